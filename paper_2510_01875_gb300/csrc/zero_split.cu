// chi0 at w = 0 on the CUDA cores for the split forms, when 0 is not on the caller's grid (the
// column S(q,0) needs), for every eta: the fallback of the tensor-core kernel of zero_tc.cu
// (taken when that kernel's 64 x 64 G tiles outnumber the SMs, or under LRT_TUNE_ZERO_SIMT).
// One extra frequency in the contraction would cost a whole 128-frequency column tile.
//
// Same Hermitian split as the contraction: with P_p = rho_p(G) rho_p*(G') and
// w_p = df_p sB/(Delta_p + i eta), RR = sum Pr wr, RI = sum Pr wi, IR = sum Pi wr, II = sum Pi wi
// give chi0(G,G') = (RR - II) + i(RI + IR) and chi0(G',G) = (RR + II) + i(RI - IR).  The work
// is 8 FP32 FMAs per (G <= G', pair) and eta with nothing to reuse across columns, so the
// kernel is bound by its shared-memory reads of the pair densities:
//  * the G set is cut into consecutive pairs (2a, 2a + 1) and a thread takes one quad of the
//    row-major list of G-pair pairs (a <= b): its four entries (2a + i, 2b + j) come from two
//    16-byte shared loads per pair p, half the shared traffic of one entry per load pair (the
//    quads on the diagonal hold three distinct entries);
//  * the pair densities of every G are staged once per 32-pair chunk with double-buffered
//    asynchronous copies, pair-major [32][N_G rounded up to even] (16-byte aligned G pairs);
//  * products and sums in packed FP32x2, partial sums over 1024 pairs flushed into FP64 sums
//    kept in shared memory (so that three blocks of 8 warps fit on an SM), then FP64 atomics.
#include "lrt_internal.h"
#include "tc_ptx.cuh"

namespace lrt {
namespace {

using namespace tcx;

constexpr int ZE = 2;              // etas per pass of an eta list
constexpr int ZL_THREADS = 256;    // one quad per thread
struct ZEtas {
  float v[64];
};

template <int ZN>   // etas per pass (1, or ZE for an eta list)
__global__ void __launch_bounds__(ZL_THREADS, 3) chi0_zero_split_kernel(
    const float2* __restrict__ rho, int gpad, const float4* __restrict__ pw, long long np,
    long long per, int nG, int nquad, int neta, int e0, double scale, double2* __restrict__ chi0,
    long long mat_stride, ZEtas etas) {
  const int nGe = (nG + 1) & ~1;          // G rows in shared memory, rounded up to even
  const int nP = nGe / 2;                 // G pairs
  extern __shared__ __align__(16) float2 zs[];
  float2* rs = zs;                        // [2][32 pairs][nGe]
  float2* ws = zs + (size_t)64 * nGe;     // [2][ZN][32] weights
  double* sums = reinterpret_cast<double*>(ws + 2 * ZN * 32);   // [4 entries][ZN][4][threads]
  const int tid = threadIdx.x;
  // this thread's quad (a, b), a <= b, of the row-major list of G-pair pairs
  int qa = -1, qb = 0;
  {
    const int idx = blockIdx.y * ZL_THREADS + tid;
    if (idx < nquad) {
      int a = 0, rem = idx;
      while (rem >= nP - a) {
        rem -= nP - a;
        ++a;
      }
      qa = a;
      qb = a + rem;
    }
  }
  const int ne = min(ZN, neta - e0);
  // packed FP32 partial sums per entry (i, j) -> 2 i + j: rr_ri = (RR, RI), ir_ii = (IR, II)
  float2 rr_ri[4][ZN], ir_ii[4][ZN];
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int e = 0; e < ZN; ++e) {
      rr_ri[t][e] = ir_ii[t][e] = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 4; ++c) sums[((t * ZN + e) * 4 + c) * ZL_THREADS + tid] = 0.0;
    }
  auto flush = [&]() {   // FP32 partial sums into the FP64 sums
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int e = 0; e < ZN; ++e) {
        double* sm = sums + (size_t)((t * ZN + e) * 4) * ZL_THREADS + tid;
        sm[0] += (double)rr_ri[t][e].x;
        sm[ZL_THREADS] += (double)rr_ri[t][e].y;
        sm[2 * ZL_THREADS] += (double)ir_ii[t][e].x;
        sm[3 * ZL_THREADS] += (double)ir_ii[t][e].y;
        rr_ri[t][e] = ir_ii[t][e] = make_float2(0.f, 0.f);
      }
  };
  const long long pb = (long long)blockIdx.x * per, pe = min(np, pb + per);
  // double-buffered chunks: the pair densities of chunk c + 1 arrive by asynchronous copies
  // while chunk c is summed
  const int nchunk = (int)((pe - pb + 31) / 32);
  auto issue = [&](int c) {
    const long long p0 = pb + 32LL * c;   // a multiple of 32: one 32-pair group of the layout
    const float2* src = rho + ((size_t)(p0 >> 5) * gpad << 5);
    const uint32_t dst = smem_u32(rs + (size_t)(c & 1) * 32 * nGe);
    for (int e = tid; e < 32 * nGe; e += ZL_THREADS) {
      const int G = e >> 5, i = e & 31;
      const bool ok = G < nG && p0 + i < pe;   // (the padding G row reads as zero)
      cp_async8(dst + (uint32_t)(i * nGe + G) * 8u, ok ? (const void*)(src + ((size_t)G << 5) + i) : (const void*)rho,
                ok ? 8u : 0u);
    }
    cp_async_commit();
  };
  if (nchunk > 0) issue(0);
  int nch = 0;
  for (int ck = 0; ck < nchunk; ++ck) {
    const long long p0 = pb + 32LL * ck;
    const float2* rb = rs + (size_t)(ck & 1) * 32 * nGe;
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
    if (qa >= 0) {
#pragma unroll 1
      for (int i = 0; i < 32; ++i) {
        float2 w[ZN];
#pragma unroll
        for (int e = 0; e < ZN; ++e) w[e] = wb[e * 32 + i];
        const float4 A = *reinterpret_cast<const float4*>(rb + (size_t)i * nGe + 2 * qa);
        const float4 B = *reinterpret_cast<const float4*>(rb + (size_t)i * nGe + 2 * qb);
        const float2 a2[2] = {make_float2(A.x, A.y), make_float2(A.z, A.w)};
        const float2 b2[2] = {make_float2(B.x, B.y), make_float2(B.z, B.w)};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float2 a = a2[t >> 1], b = b2[t & 1];
          // a conj(b) = b.x (a.x, a.y) + b.y (a.y, -a.x)
          const float2 P = __ffma2_rn(make_float2(b.x, b.x), a,
                                      __fmul2_rn(make_float2(b.y, b.y), make_float2(a.y, -a.x)));
#pragma unroll
          for (int e = 0; e < ZN; ++e) {
            rr_ri[t][e] = __ffma2_rn(make_float2(P.x, P.x), w[e], rr_ri[t][e]);
            ir_ii[t][e] = __ffma2_rn(make_float2(P.y, P.y), w[e], ir_ii[t][e]);
          }
        }
      }
    }
    if (++nch == 32) {   // FP32 partial sums over 1024 pairs, then into FP64
      nch = 0;
      flush();
    }
  }
  flush();
  if (qa < 0) return;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int G = 2 * qa + (t >> 1), Gp = 2 * qb + (t & 1);
    // padding G, and the repeated lower entry of a diagonal quad
    if (G >= nG || Gp >= nG || G > Gp) continue;
    for (int e = 0; e < ne; ++e) {
      const double* sm = sums + (size_t)((t * ZN + e) * 4) * ZL_THREADS + tid;
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
  bool done = false;
  if (!c->zero_simt) LRT_TRY(launch_zero_tc(c, q, rho, sB, s, &done));
  if (done) return LRT_OK;
  const int nG = q.nG;
  const long long mat = (long long)nG * nG;
  double2* base = q.chi0 + (size_t)c->hcol * mat;
  LRT_CUDA(cudaMemset2DAsync(base, (size_t)c->nwi * mat * sizeof(double2), 0, (size_t)mat * sizeof(double2),
                             c->neta, s));
  int dev = 0, nsm = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int nGe = (nG + 1) & ~1, nP = nGe / 2;
  const int nquad = nP * (nP + 1) / 2;
  const int ntile = (nquad + ZL_THREADS - 1) / ZL_THREADS;
  // about six blocks per SM in all (three resident at a time), each over one range of pairs
  // (a multiple of 32)
  long long nsplit = std::max<long long>(1, (6LL * nsm + ntile - 1) / ntile);
  long long per = (c->np + nsplit - 1) / nsplit;
  per = (per + 31) / 32 * 32;
  nsplit = (c->np + per - 1) / per;
  const double rs = split_rho_scale(c->precision);
  const double scale = 2.0 / (c->nk * c->volume) / (rs * rs * (double)sB);
  ZEtas E{};   // the etas travel as a kernel argument (at most 64)
  for (int j = 0; j < c->neta; ++j) E.v[j] = (float)c->etas[j];
  const bool list = c->neta > 1;
  const int zn = list ? ZE : 1;
  const size_t smem = ((size_t)64 * nGe + (size_t)zn * 64) * sizeof(float2) +
                      (size_t)4 * zn * 4 * ZL_THREADS * sizeof(double);
  auto k1 = chi0_zero_split_kernel<1>;
  auto k2 = chi0_zero_split_kernel<ZE>;
  LRT_CUDA(cudaFuncSetAttribute(list ? k2 : k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int e0 = 0; e0 < c->neta; e0 += ZE) {
    (list ? k2 : k1)<<<dim3((unsigned)nsplit, (unsigned)ntile), ZL_THREADS, smem, s>>>(
        (const float2*)rho, c->rho_gpad, q.sp.pw, c->np, per, nG, nquad, c->neta, e0, scale, base,
        (long long)c->nwi * mat, E);
    count_launch(c);
    LRT_CUDA(cudaGetLastError());
    if (!list) break;
  }
  return LRT_OK;
}

}  // namespace lrt
