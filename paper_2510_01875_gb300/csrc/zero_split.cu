// chi0 at w = 0 on the CUDA cores for the split forms, when 0 is not on the caller's grid.
#include "lrt_internal.h"
#include "tc_ptx.cuh"

namespace lrt {
namespace {

using namespace tcx;

// chi0 at w = 0 when 0 is not on the caller's grid (the column S(q,0) needs), for every eta,
// on the CUDA cores instead of a tensor tile of its own (one extra frequency would cost a whole
// 128-frequency column tile of the contraction).  Same Hermitian split as the contraction:
// with P_p = rho_p(G) rho_p*(G') and w_p = df_p sB/(Delta_p + i eta), RR = sum Pr wr,
// RI = sum Pr wi, IR = sum Pi wr, II = sum Pi wi give chi0(G,G') = (RR - II) + i(RI + IR) and
// chi0(G',G) = (RR + II) + i(RI - IR).  FP32 products and per-thread FP32 partial sums over
// 1024 pairs, flushed into FP64 (round-to-nearest, so unbiased), then FP64 atomics into chi0.
// Grid (pair range, tile of the G <= G' list); block 256, each thread E entries of the
// row-major list of G <= G' pairs (no padding but in the last tile), the pair densities of
// every G staged once per 32-pair chunk; ZN etas per pass.  8 FP32 FMAs per (entry, pair)
// and eta: the work is that of the one frequency, so nothing is reused across columns.
constexpr int ZE = 2;    // etas per pass of an eta list
constexpr int ZL_THREADS = 1024;
struct ZEtas {
  float v[64];
};
// Shared memory: two 32-pair chunks of the pair densities of every G, [32 pairs][nG] (pair-major,
// so the lanes of a warp, which hold consecutive G', read without bank conflicts), their
// weights [2][ZN][32], and the FP64 sums [E ZN 4][ZL_THREADS] (in shared memory rather than
// registers, so that 32 warps fit on an SM to hide the shared-memory and FMA latencies).
template <int ZN, int E>   // etas per pass (1, or ZE for an eta list); G <= G' pairs per thread
__global__ void __launch_bounds__(ZL_THREADS, 1) chi0_zero_split_kernel(
    const float2* __restrict__ rho, int gpad, const float4* __restrict__ pw, long long np,
    long long per, int nG, int ngg, int neta, int e0, double scale, double2* __restrict__ chi0,
    long long mat_stride, ZEtas etas) {
  extern __shared__ __align__(16) float2 zs[];
  float2* rs = zs;
  float2* ws = zs + (size_t)64 * nG;
  double* sums = reinterpret_cast<double*>(ws + 2 * ZN * 32);
  const int tid = threadIdx.x;
  int ga[E], gb[E];
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int idx = blockIdx.y * (ZL_THREADS * E) + k * ZL_THREADS + tid;
    ga[k] = -1;
    gb[k] = 0;
    if (idx < ngg) {   // entry idx of the row-major list of (G, G'), G <= G'
      int G = 0, rem = idx;
      while (rem >= nG - G) {
        rem -= nG - G;
        ++G;
      }
      ga[k] = G;
      gb[k] = G + rem;
    }
  }
  const int ne = min(ZN, neta - e0);
  // FP32 partial sums as packed pairs: rr_ri = (RR, RI), ir_ii = (IR, II)
  float2 rr_ri[E][ZN], ir_ii[E][ZN];
#pragma unroll
  for (int k = 0; k < E; ++k)
#pragma unroll
    for (int e = 0; e < ZN; ++e) {
      rr_ri[k][e] = ir_ii[k][e] = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 4; ++c) sums[((k * ZN + e) * 4 + c) * ZL_THREADS + tid] = 0.0;
    }
  auto flush = [&]() {   // FP32 partial sums into the FP64 sums
#pragma unroll
    for (int k = 0; k < E; ++k)
#pragma unroll
      for (int e = 0; e < ZN; ++e) {
        double* sm = sums + (size_t)((k * ZN + e) * 4) * ZL_THREADS + tid;
        sm[0] += (double)rr_ri[k][e].x;
        sm[ZL_THREADS] += (double)rr_ri[k][e].y;
        sm[2 * ZL_THREADS] += (double)ir_ii[k][e].x;
        sm[3 * ZL_THREADS] += (double)ir_ii[k][e].y;
        rr_ri[k][e] = ir_ii[k][e] = make_float2(0.f, 0.f);
      }
  };
  const long long pb = (long long)blockIdx.x * per, pe = min(np, pb + per);
  // double-buffered chunks: the pair densities of chunk c + 1 arrive by asynchronous copies
  // while chunk c is summed
  const int nchunk = (int)((pe - pb + 31) / 32);
  auto issue = [&](int c) {
    const long long p0 = pb + 32LL * c;   // a multiple of 32: one 32-pair group of the layout
    const float2* src = rho + ((size_t)(p0 >> 5) * gpad << 5);
    const uint32_t dst = smem_u32(rs + (size_t)(c & 1) * 32 * nG);
    for (int e = tid; e < 32 * nG; e += ZL_THREADS) {
      const int G = e >> 5, i = e & 31;
      const bool ok = p0 + i < pe;
      cp_async8(dst + (uint32_t)(i * nG + G) * 8u, ok ? (const void*)(src + ((size_t)G << 5) + i) : (const void*)rho,
                ok ? 8u : 0u);
    }
    cp_async_commit();
  };
  if (nchunk > 0) issue(0);
  int nch = 0;
  for (int ck = 0; ck < nchunk; ++ck) {
    const long long p0 = pb + 32LL * ck;
    float2* rb = rs + (size_t)(ck & 1) * 32 * nG;
    float2* wb = ws + (size_t)(ck & 1) * ZN * 32;
    cp_async_wait_all();
    if (tid < 32) {
      const long long p = p0 + tid;
      const float4 q = p < pe ? pw[p] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float x = q.x + q.y;
#pragma unroll
      for (int e = 0; e < ZN; ++e) {
        float2 w = make_float2(0.f, 0.f);
        if (p < pe && e < ne) {
          const float eta = etas.v[e0 + e];
          const float r = 1.0f / (x * x + eta * eta);
          w = make_float2(q.z * x * r, -q.z * eta * r);   // df sB / (x + i eta)
        }
        wb[e * 32 + tid] = w;
      }
    }
    // chunk ck is complete for every thread, and the other buffer's readers (chunk ck - 1) are
    // done
    __syncthreads();
    if (ck + 1 < nchunk) issue(ck + 1);
#pragma unroll 2
    for (int i = 0; i < 32; ++i) {
      float2 w[ZN];
#pragma unroll
      for (int e = 0; e < ZN; ++e) w[e] = wb[e * 32 + i];
#pragma unroll
      for (int k = 0; k < E; ++k) {
        if (ga[k] < 0) continue;
        const float2 a = rb[i * nG + ga[k]], b = rb[i * nG + gb[k]];
        // a conj(b) = b.x (a.x, a.y) + b.y (a.y, -a.x), in packed FP32x2
        const float2 P = __ffma2_rn(make_float2(b.x, b.x), a,
                                    __fmul2_rn(make_float2(b.y, b.y), make_float2(a.y, -a.x)));
#pragma unroll
        for (int e = 0; e < ZN; ++e) {
          rr_ri[k][e] = __ffma2_rn(make_float2(P.x, P.x), w[e], rr_ri[k][e]);
          ir_ii[k][e] = __ffma2_rn(make_float2(P.y, P.y), w[e], ir_ii[k][e]);
        }
      }
    }
    if (++nch == 32) {   // FP32 partial sums over 1024 pairs, then into FP64
      nch = 0;
      flush();
    }
  }
  flush();
#pragma unroll
  for (int k = 0; k < E; ++k) {
    if (ga[k] < 0) continue;
    const int G = ga[k], Gp = gb[k];
    for (int e = 0; e < ne; ++e) {
      const double* sm = sums + (size_t)((k * ZN + e) * 4) * ZL_THREADS + tid;
      const double RR = sm[0], RI = sm[ZL_THREADS], IR = sm[2 * ZL_THREADS], II = sm[3 * ZL_THREADS];
      double2* m = chi0 + (size_t)(e0 + e) * mat_stride;
      atomicAdd(&m[(size_t)G * nG + Gp].x, scale * (RR - II));
      atomicAdd(&m[(size_t)G * nG + Gp].y, scale * (RI + IR));
      if (G != Gp) {
        atomicAdd(&m[(size_t)Gp * nG + G].x, scale * (RR + II));
        atomicAdd(&m[(size_t)Gp * nG + G].y, scale * (RI - IR));
      }
    }
  }
}

}  // namespace

lrt_status launch_zero_split(const lrt_ctx* c, QData& q, const void* rho, float sB, cudaStream_t s) {
  if (c->hcol != c->nw) return LRT_OK;   // w = 0 is on the grid: a tensor column
  const int nG = q.nG;
  const long long mat = (long long)nG * nG;
  double2* base = q.chi0 + (size_t)c->hcol * mat;
  LRT_CUDA(cudaMemset2DAsync(base, (size_t)c->nwi * mat * sizeof(double2), 0, (size_t)mat * sizeof(double2),
                             c->neta, s));
  int dev = 0, nsm = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int ngg = nG * (nG + 1) / 2;
  const bool list = c->neta > 1;
  constexpr int NE = 2;   // entries per thread (both pass widths)
  const int per_block = ZL_THREADS * NE;
  const int ntile = (ngg + per_block - 1) / per_block;
  // about four blocks per SM in all (two resident at a time), each over one range of pairs
  // (a multiple of 32)
  long long nsplit = std::max<long long>(1, (4LL * nsm + ntile - 1) / ntile);
  long long per = (c->np + nsplit - 1) / nsplit;
  per = (per + 31) / 32 * 32;
  nsplit = (c->np + per - 1) / per;
  const double rs = split_rho_scale(c->precision);
  const double scale = 2.0 / (c->nk * c->volume) / (rs * rs * (double)sB);
  ZEtas E{};   // the etas travel as a kernel argument (at most 64)
  for (int j = 0; j < c->neta; ++j) E.v[j] = (float)c->etas[j];
  const int zn = list ? ZE : 1;
  const size_t smem = ((size_t)64 * nG + (size_t)zn * 64) * sizeof(float2) +
                      (size_t)NE * zn * 4 * ZL_THREADS * sizeof(double);
  auto k1 = chi0_zero_split_kernel<1, NE>;
  auto k2 = chi0_zero_split_kernel<ZE, NE>;
  LRT_CUDA(cudaFuncSetAttribute(list ? k2 : k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int e0 = 0; e0 < c->neta; e0 += ZE) {
    (list ? k2 : k1)<<<dim3((unsigned)nsplit, (unsigned)ntile), ZL_THREADS, smem, s>>>(
        (const float2*)rho, c->rho_gpad, q.sp.pw, c->np, per, nG, ngg, c->neta, e0, scale, base,
        (long long)c->nwi * mat, E);
    count_launch(c);
    LRT_CUDA(cudaGetLastError());
    if (!list) break;
  }
  return LRT_OK;
}

}  // namespace lrt
