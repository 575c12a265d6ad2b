// Adler-Wiser chi0 in FP64 on the CUDA cores:
//   chi0_GG'(w) = (2/(N_k Omega)) sum_p rho_p(G) rho_p*(G') df_p / (w + Delta_p + i eta).
// With P_p = rho_p(G) rho_p*(G') = Pr + i Pi and w_p = wr + i wi, the four real sums
//   RR = sum Pr wr, RI = sum Pr wi, IR = sum Pi wr, II = sum Pi wi
// give both chi0(G,G') = (RR - II) + i(RI + IR) and chi0(G',G) = (RR + II) + i(RI - IR)
// (P_p(G',G) = conj P_p(G,G')), so only G <= G' is accumulated: 4 real FMAs per
// (G <= G', w, p), i.e. 4 flops per complex MAC of the full sum.
//
// The FP64 units are the only limit here (on this part they retire two FMAs per clock per SM,
// far below the shared-memory and L2 rates), so the kernel is laid out to spend as few FP64
// instructions as possible beyond those 4 FMAs:
//  * a block tile is 64 consecutive entries of the list of (G <= G') pairs (row-major upper
//    triangle, so only the last tile has padding) x 64 frequencies x a range of pairs (split K);
//  * per chunk of 16 pairs the block forms P_p for its 64 G pairs (4 FP64 operations each,
//    shared by 64 frequencies) and w_p(w) for its 64 frequencies (one division and five
//    operations each, shared by 64 G pairs) in shared memory; neither is stored in global memory;
//  * each thread then accumulates 2 G pairs x 8 frequencies (64 FMAs per pair p, all
//    independent), warp-uniform frequencies, so a warp whose frequencies lie past the grid
//    skips the work.
// Partial sums go to chi0 with FP64 atomics.
#include "lrt_internal.h"

namespace lrt {
namespace {

constexpr int TGG = 64;   // (G <= G') pairs per tile
constexpr int TW = 64;    // frequencies per tile
constexpr int PC = 16;    // pairs per chunk
constexpr int NT = 256;   // threads: warp w takes frequencies 8 w .. 8 w + 7, lane l G pairs l, l + 32

__global__ void __launch_bounds__(NT, 1) chi0_fp64_kernel(
    const double2* __restrict__ rho, const double* __restrict__ delta,
    const double* __restrict__ df, const double* __restrict__ freqs, int nwi, int nG, int ngp,
    int64_t np, int64_t ld, double eta, double pref, int64_t p_per_split,
    double2* __restrict__ chi0) {
  __shared__ double2 Ps[PC][TGG + 1];
  __shared__ double2 Ws[PC][TW];
  __shared__ int2 gp_s[TGG];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int w0 = blockIdx.y * TW;
  const int64_t pbeg = (int64_t)blockIdx.z * p_per_split;
  const int64_t pend = min(np, pbeg + p_per_split);
  if (tid < TGG) {
    // entry e of the row-major list of (G, G'), G <= G'
    const int e = blockIdx.x * TGG + tid;
    int2 g = make_int2(-1, -1);
    if (e < ngp) {
      int G = 0, rem = e;
      while (rem >= nG - G) {
        rem -= nG - G;
        ++G;
      }
      g = make_int2(G, G + rem);
    }
    gp_s[tid] = g;
  }
  __syncthreads();
  const bool active = w0 + 8 * warp < nwi;   // warp-uniform
  double RR[2][8], RI[2][8], IR[2][8], II[2][8];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int t = 0; t < 8; ++t) RR[i][t] = RI[i][t] = IR[i][t] = II[i][t] = 0.0;
  const double eta2 = eta * eta;
  for (int64_t p0 = pbeg; p0 < pend; p0 += PC) {
    // P_p(G, G') of the tile's G pairs (lanes along p: coalesced reads of the rho rows)
    for (int e = tid; e < TGG * PC; e += NT) {
      const int p = e % PC, g = e / PC;
      const int64_t pp = p0 + p;
      const int2 gg = gp_s[g];
      double2 v = make_double2(0.0, 0.0);
      if (pp < pend && gg.x >= 0) {
        const double2 x = rho[(size_t)gg.x * ld + pp], y = rho[(size_t)gg.y * ld + pp];
        v = make_double2(x.x * y.x + x.y * y.y, x.y * y.x - x.x * y.y);
      }
      Ps[p][g] = v;
    }
    // w_p(w) = df_p (x - i eta)/(x^2 + eta^2), x = w + Delta_p
    for (int e = tid; e < TW * PC; e += NT) {
      const int p = e % PC, w = e / PC;
      const int64_t pp = p0 + p;
      double2 v = make_double2(0.0, 0.0);
      if (pp < pend && w0 + w < nwi) {
        const double x = freqs[w0 + w] + delta[pp];
        const double s = df[pp] / fma(x, x, eta2);
        v = make_double2(s * x, -s * eta);
      }
      Ws[p][w] = v;
    }
    __syncthreads();
    if (active) {
#pragma unroll 2
      for (int p = 0; p < PC; ++p) {
        const double2 a0 = Ps[p][lane], a1 = Ps[p][lane + 32];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const double2 w = Ws[p][8 * warp + t];
          RR[0][t] = fma(a0.x, w.x, RR[0][t]);
          RI[0][t] = fma(a0.x, w.y, RI[0][t]);
          IR[0][t] = fma(a0.y, w.x, IR[0][t]);
          II[0][t] = fma(a0.y, w.y, II[0][t]);
          RR[1][t] = fma(a1.x, w.x, RR[1][t]);
          RI[1][t] = fma(a1.x, w.y, RI[1][t]);
          IR[1][t] = fma(a1.y, w.x, IR[1][t]);
          II[1][t] = fma(a1.y, w.y, II[1][t]);
        }
      }
    }
    __syncthreads();
  }
  if (!active) return;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int2 gg = gp_s[lane + 32 * i];
    if (gg.x < 0) continue;
    const int G = gg.x, Gp = gg.y;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int w = w0 + 8 * warp + t;
      if (w >= nwi) continue;
      double2* base = chi0 + (size_t)w * nG * nG;
      atomicAdd(&base[(size_t)G * nG + Gp].x, pref * (RR[i][t] - II[i][t]));
      atomicAdd(&base[(size_t)G * nG + Gp].y, pref * (RI[i][t] + IR[i][t]));
      if (G != Gp) {
        atomicAdd(&base[(size_t)Gp * nG + G].x, pref * (RR[i][t] + II[i][t]));
        atomicAdd(&base[(size_t)Gp * nG + G].y, pref * (RI[i][t] - IR[i][t]));
      }
    }
  }
}

}  // namespace

lrt_status launch_chi0_fp64(const lrt_ctx* c, QData& q, cudaStream_t s) {
  const int ngp = q.nG * (q.nG + 1) / 2;
  const int ngt = (ngp + TGG - 1) / TGG;
  const int nwt = (c->nwi + TW - 1) / TW;
  const int64_t tiles = (int64_t)ngt * nwt;
  int dev = 0, nsm = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // K splits: at least ~4 blocks per SM, and among the counts up to twice that the one whose
  // last wave of blocks (one block per SM) is fullest
  const int64_t maxsplit = std::max<int64_t>(1, (c->np + PC - 1) / PC);
  const int64_t lo = std::min<int64_t>(maxsplit, std::max<int64_t>(1, (4 * nsm + tiles - 1) / tiles));
  const int64_t hi = std::min<int64_t>(std::min<int64_t>(maxsplit, 2 * lo), 65535);
  int64_t split = lo;
  double best = 0.0;
  for (int64_t sp = lo; sp <= hi; ++sp) {
    const int64_t blocks = tiles * sp;
    const double fill = (double)blocks / (double)(((blocks + nsm - 1) / nsm) * nsm);
    if (fill > best + 1e-9) {
      best = fill;
      split = sp;
    }
  }
  int64_t per = (c->np + split - 1) / split;
  per = (per + PC - 1) / PC * PC;
  split = (c->np + per - 1) / per;
  LRT_CUDA(cudaMemsetAsync(q.chi0, 0, (size_t)ncol(c) * q.nG * q.nG * sizeof(double2), s));
  dim3 grid(ngt, nwt, (unsigned)split);
  double pref = 2.0 / (c->nk * c->volume);
  // one launch per broadening of the eta list, into that eta's block of chi0
  for (int j = 0; j < c->neta; ++j) {
    TimedLaunch tl(c, &c->ev_chi0, s);
    chi0_fp64_kernel<<<grid, NT, 0, s>>>((const double2*)c->dw.rho, c->dw.delta, c->dw.df,
                                         c->dw.freqs, c->nwi, q.nG, ngp, c->np, c->rho_ld,
                                         c->etas[j], pref, per,
                                         q.chi0 + (size_t)j * c->nwi * q.nG * q.nG);
    count_launch(c);
    LRT_CUDA(cudaGetLastError());
  }
  if (c->profiling) c->timed_cmac += (double)q.nG * q.nG * c->nw * (double)c->np * c->neta;
  return LRT_OK;
}

}  // namespace lrt
