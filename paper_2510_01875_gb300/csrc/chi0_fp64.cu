// Adler-Wiser chi0 in FP64 on the CUDA cores:
//   chi0_GG'(w) = (2/(N_k Omega)) sum_p rho_p(G) rho_p*(G') df_p / (w + Delta_p + i eta).
// With P_p = rho_p(G) rho_p*(G') = Pr + i Pi and w_p = wr + i wi, the four real sums
//   RR = sum Pr wr, RI = sum Pr wi, IR = sum Pi wr, II = sum Pi wi
// give both chi0(G,G') = (RR - II) + i(RI + IR) and chi0(G',G) = (RR + II) + i(RI - IR)
// (P_p(G',G) = conj P_p(G,G')), so only G <= G' is accumulated: 4 real FMAs per
// (G <= G', w, p), i.e. 4 flops per complex MAC of the full sum.
//
// Block: an 8 x 8 block pair (I <= J) of G values x 32 frequencies x a range of pairs (split
// K); partial sums go to chi0 with FP64 atomics.  The weights w_p(w) are generated in shared
// memory per chunk of 32 pairs and never stored in global memory.
#include "lrt_internal.h"

namespace lrt {
namespace {

constexpr int GB = 8;    // G per block side
constexpr int WT = 32;   // frequencies per block
constexpr int PC = 32;   // pairs per chunk

__global__ void __launch_bounds__(256) chi0_fp64_kernel(
    const double2* __restrict__ rho, const double* __restrict__ delta,
    const double* __restrict__ df, const double* __restrict__ freqs, int nwi, int nG,
    int64_t np, int64_t ld, double eta, double pref, int nblk, int64_t p_per_split,
    double2* __restrict__ chi0) {
  __shared__ double2 rI[PC][GB];
  __shared__ double2 rJ[PC][GB];
  __shared__ double2 ws[PC][WT];
  // block pair (I, J), I <= J, from the linear index
  int bp = blockIdx.x, I = 0;
  while (bp >= nblk - I) {
    bp -= nblk - I;
    ++I;
  }
  const int J = I + bp;
  const int w0 = blockIdx.y * WT;
  const int64_t pbeg = (int64_t)blockIdx.z * p_per_split;
  const int64_t pend = min(np, pbeg + p_per_split);
  const int tid = threadIdx.x;
  const int gi = (tid & 63) >> 3, gj = tid & 7, wg = tid >> 6;
  double RR[8], RI[8], IR[8], II[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) RR[t] = RI[t] = IR[t] = II[t] = 0.0;
  for (int64_t p0 = pbeg; p0 < pend; p0 += PC) {
    {
      int p = tid & 31, g = tid >> 5;
      int64_t pp = p0 + p;
      int GI = I * GB + g, GJ = J * GB + g;
      double2 z = make_double2(0.0, 0.0);
      rI[p][g] = (pp < pend && GI < nG) ? rho[(size_t)GI * ld + pp] : z;
      rJ[p][g] = (pp < pend && GJ < nG) ? rho[(size_t)GJ * ld + pp] : z;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + 256 * r;
      int p = e & 31, w = e >> 5;
      int64_t pp = p0 + p;
      double2 v = make_double2(0.0, 0.0);
      if (pp < pend && w0 + w < nwi) {
        double x = freqs[w0 + w] + delta[pp];
        double s = df[pp] / (x * x + eta * eta);
        v = make_double2(s * x, -s * eta);
      }
      ws[p][w] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int p = 0; p < PC; ++p) {
      double2 a = rI[p][gi], b = rJ[p][gj];
      double pr = a.x * b.x + a.y * b.y;
      double pi = a.y * b.x - a.x * b.y;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        double2 w = ws[p][wg * 8 + t];
        RR[t] = fma(pr, w.x, RR[t]);
        RI[t] = fma(pr, w.y, RI[t]);
        IR[t] = fma(pi, w.x, IR[t]);
        II[t] = fma(pi, w.y, II[t]);
      }
    }
    __syncthreads();
  }
  const int G = I * GB + gi, Gp = J * GB + gj;
  if (G >= nG || Gp >= nG) return;
  if (I == J && gi > gj) return;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    int w = w0 + wg * 8 + t;
    if (w >= nwi) continue;
    double2* base = chi0 + (size_t)w * nG * nG;
    atomicAdd(&base[(size_t)G * nG + Gp].x, pref * (RR[t] - II[t]));
    atomicAdd(&base[(size_t)G * nG + Gp].y, pref * (RI[t] + IR[t]));
    if (G != Gp) {
      atomicAdd(&base[(size_t)Gp * nG + G].x, pref * (RR[t] + II[t]));
      atomicAdd(&base[(size_t)Gp * nG + G].y, pref * (RI[t] - IR[t]));
    }
  }
}

}  // namespace

lrt_status launch_chi0_fp64(const lrt_ctx* c, QData& q, cudaStream_t s) {
  int nblk = (q.nG + GB - 1) / GB;
  int npairs = nblk * (nblk + 1) / 2;
  int nwt = (c->nwi + WT - 1) / WT;
  int64_t tiles = (int64_t)npairs * nwt;
  // enough K splits for ~8 blocks per SM, each split a multiple of the chunk
  int64_t want = (8 * 152 + tiles - 1) / tiles;
  int64_t maxsplit = (c->np + PC - 1) / PC;
  int64_t split = want < 1 ? 1 : (want > maxsplit ? maxsplit : want);
  if (split > 65535) split = 65535;
  int64_t per = (c->np + split - 1) / split;
  per = (per + PC - 1) / PC * PC;
  split = (c->np + per - 1) / per;
  LRT_CUDA(cudaMemsetAsync(q.chi0, 0, (size_t)ncol(c) * q.nG * q.nG * sizeof(double2), s));
  dim3 grid(npairs, nwt, (unsigned)split);
  double pref = 2.0 / (c->nk * c->volume);
  // one launch per broadening of the eta list, into that eta's block of chi0
  for (int j = 0; j < c->neta; ++j) {
    TimedLaunch tl(c, &c->ev_chi0, s);
    chi0_fp64_kernel<<<grid, 256, 0, s>>>((const double2*)c->dw.rho, c->dw.delta, c->dw.df,
                                          c->dw.freqs, c->nwi, q.nG, c->np, c->rho_ld, c->etas[j],
                                          pref, nblk, per,
                                          q.chi0 + (size_t)j * c->nwi * q.nG * q.nG);
    count_launch(c);
    LRT_CUDA(cudaGetLastError());
  }
  if (c->profiling) c->timed_cmac += (double)q.nG * q.nG * c->nw * (double)c->np * c->neta;
  return LRT_OK;
}

}  // namespace lrt
