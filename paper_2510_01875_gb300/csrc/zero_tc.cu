// chi0 at w = 0 for the split forms on the 5th-generation tensor cores (tcgen05, one CTA per
// SM), when 0 is not on the caller's grid (the column S(q,0) needs), one eta per launch.
//
// At a single frequency the contraction has no frequency axis to reuse the pair products
// over, so it is run in the other order: with u_p(G') = rho_p*(G') w_p and
// w_p = df_p / (Delta_p + i eta),
//   chi0_GG'(0) = pref sum_p rho_p(G) u_p(G')
// is one complex GEMM over the pairs, O(N_G) operand values per pair instead of O(N_G^2).  As
// a real GEMM, rows (G, Re|Im of rho) against columns (G', Re|Im of u):
//   C_ab(G, G') = sum_p rho_a(G) u_b(G'),  chi0 = (C_rr - C_ii) + i (C_ri + C_ir).
// Tiles are 64 G x 64 G' (M = N = 128) over the pairs, FP16 x 3 (or BF16 x 3) with FP32
// tensor-memory accumulators like the contraction: rho carries the split path's power-of-two
// scale r, u = conj(rho) w / r with w = df sB / (Delta + i eta) as in the contraction's
// columns, so both operands stay in the FP16 range.
//
// The kernel reads every pair density once per tile row/column block and does little else, so
// it is bound by that HBM read.  Per 32-pair stage: a loader copies the stage's rho rows of the
// tile's two 64-G blocks (one or two contiguous bulk copies of the blocked layout
// rho[p/32][G][p%32]) and the 32 pair weights into a ring; 8 producer warps (lane = pair) form
// w, the A rows (rho) and B columns (u), split them into hi and lo parts and write the
// MN-major 128-byte-swizzled tiles; one thread issues A_hi B_hi + A_hi B_lo + A_lo B_hi.
// Every 64 stages (2048 pairs) the accumulator (two alternate in tensor memory) is drained by
// four epilogue warps into this CTA's own FP64 partial sums in global memory (plain
// read-add-write: each thread owns one row); a second kernel adds the partial sums of the
// CTAs of each tile into chi0.  The CTAs of the grid are dealt to the tiles round-robin and
// split each tile's pairs evenly.  Every wait is bounded; on expiry bit 2 of the status word is
// set and the kernel drains and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "lrt_internal.h"
#include "tc_ptx.cuh"

namespace lrt {
namespace {

using namespace tcx;

constexpr int ZG = 64;                       // G per tile side
constexpr int ZM = 2 * ZG;                   // MMA M = N = 128 (G, Re|Im)
constexpr int ZK = 32;                       // pairs (K) per stage
constexpr int ZNS = 3;                       // operand stages
constexpr int ZNR = 3;                       // ring stages (rho rows + pair weights)
constexpr int ZA_BYTES = ZM * ZK * 2;        // 8 KB, one 16-bit operand tile
constexpr int ZSTAGE = 4 * ZA_BYTES;         // A hi, A lo, B hi, B lo: 32 KB
constexpr int ZSBO = (ZM / 64) * 1024;       // bytes between 8-pair groups
constexpr int ZRB = ZG * ZK * 8;             // one 64-G block of one stage: 16 KB
constexpr int ZR_PW = 2 * ZRB;               // pair weights after the two blocks
constexpr int ZR_STAGE = ZR_PW + ZK * 16;
constexpr int ZW_MMA = 8, ZW_LOAD = 9;       // producers 0..7, epilogue 10..13
constexpr int ZTHREADS = 14 * 32;
constexpr int ZPERIOD = 64;                  // stages per FP32 accumulation period
constexpr size_t ZSMEM = (size_t)ZNS * ZSTAGE + (size_t)ZNR * ZR_STAGE + 1024;

struct ZParams {
  const float2* rho;          // blocked [.. / 32][gpad][32]
  const float4* pw;           // {Delta_hi, Delta_lo, df sB, 0} per pair, zero padding
  double* part;               // [gridDim.x][ZM columns][ZM rows] FP64 partial sums
  int* status;
  long long nstage;           // 32-pair stages (the pairs rounded up to 32)
  int gpad, ntile, rt;        // rows of the layout, tiles (rt x rt), 64-G blocks
  float eta, inv_r;           // this launch's eta; 1 / (the pair densities' scale)
};

// Tile and stage range of CTA b: tile b % ntile; the CTAs of a tile split its stages in
// ZPERIOD multiples.
struct ZWork {
  int I, J;
  long long s0, s1;
};
__host__ __device__ __forceinline__ ZWork zwork(const ZParams& P, int b, int grid) {
  ZWork w;
  const int t = b % P.ntile;
  w.I = t / P.rt;
  w.J = t % P.rt;
  const int n = (grid - t + P.ntile - 1) / P.ntile;   // CTAs of tile t
  const int k = b / P.ntile;                          // this CTA's share
  const long long nper = (P.nstage + ZPERIOD - 1) / ZPERIOD;
  const long long per = (nper + n - 1) / n;
  const long long a = (long long)k * per * ZPERIOD, b2 = a + per * ZPERIOD;
  w.s0 = a < P.nstage ? a : P.nstage;
  w.s1 = b2 < P.nstage ? b2 : P.nstage;
  return w;
}

template <bool BF>
__global__ void __launch_bounds__(ZTHREADS, 1) chi0_zero_tc_kernel(ZParams P) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[ZNS], empty[ZNS], rfull[ZNR], rempty[ZNR];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], final_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t rbase = base + ZNS * ZSTAGE;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ZNS; ++s) {
      mbar_init(&full[s], 8);
      mbar_init(&empty[s], 1);
    }
    for (int r = 0; r < ZNR; ++r) {
      mbar_init(&rfull[r], 1);
      mbar_init(&rempty[r], 8);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(&final_bar, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == ZW_MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(2 * ZM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  const ZWork W = zwork(P, blockIdx.x, gridDim.x);
  const int nst = (int)(W.s1 - W.s0);
  const int rows_i = min(ZG, P.gpad - ZG * W.I), rows_j = min(ZG, P.gpad - ZG * W.J);
  const uint32_t jo = W.I == W.J ? 0u : (uint32_t)ZRB;   // ring offset of the G' rows

  if (warp < 8) {
    // ---------------- producers: A chunks 2 w, 2 w + 1 (rho of G 8 w .. 8 w + 7 of block I),
    // B chunks 2 w, 2 w + 1 (u of G' 8 w .. 8 w + 7 of block J); lane = pair ----------------
    const float eta = P.eta, eta2 = P.eta * P.eta;
    uint32_t it = 0;
    for (int st_ = 0; st_ < nst; ++st_, ++it) {
      const int s = it % ZNS, r = it % ZNR;
      if (!__all_sync(0xffffffffu, mbar_wait(&rfull[r], (it / ZNR) & 1, &abort_s, P.status))) break;
      if (!__all_sync(0xffffffffu, mbar_wait(&empty[s], ((it / ZNS) & 1) ^ 1, &abort_s, P.status))) break;
      const uint32_t ring = rbase + r * ZR_STAGE + stage_token();
      const uint32_t sst = base + s * ZSTAGE;
      // w = df sB / (Delta + i eta), over r so that u = conj(rho) w stays in the FP16 range
      const float4 pw = lds_f4(ring + ZR_PW + lane * 16);
      const float x = pw.x + pw.y;
      const float rd = rcp_approx(__fmaf_rn(x, x, eta2));
      const float wr = pw.z * P.inv_r * x * rd, wi = -pw.z * P.inv_r * eta * rd;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = 2 * warp + h;   // chunk: local G 4 c .. 4 c + 3
        float va[8], vb[8];
        if (4 * c < rows_i) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float2 a = lds_f2(ring + (uint32_t)((4 * c + j) * ZK * 8) + lane * 8);
            va[2 * j] = a.x;
            va[2 * j + 1] = a.y;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) va[j] = 0.f;
        }
        if (4 * c < rows_j) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float2 b = lds_f2(ring + jo + (uint32_t)((4 * c + j) * ZK * 8) + lane * 8);
            vb[2 * j] = __fmaf_rn(b.x, wr, b.y * wi);       // Re conj(rho) w
            vb[2 * j + 1] = __fmaf_rn(b.x, wi, -b.y * wr);  // Im
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) vb[j] = 0.f;
        }
        const uint32_t off = mn_chunk(lane, c, ZSBO);
        uint4 hi, lo;
        Pack<BF>::split(va, hi, lo);
        st_shared_v4(sst + off, hi);
        st_shared_v4(sst + ZA_BYTES + off, lo);
        Pack<BF>::split(vb, hi, lo);
        st_shared_v4(sst + 2 * ZA_BYTES + off, hi);
        st_shared_v4(sst + 3 * ZA_BYTES + off, lo);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&full[s]);
        mbar_arrive(&rempty[r]);
      }
    }
  } else if (warp == ZW_LOAD) {
    // ---------------- loader: rho rows of blocks I and J and the pair weights ----------------
    if (lane == 0) {
      const uint32_t bi = (uint32_t)rows_i * ZK * 8, bj = W.I == W.J ? 0u : (uint32_t)rows_j * ZK * 8;
      uint32_t it = 0;
      for (int st_ = 0; st_ < nst; ++st_, ++it) {
        const int r = it % ZNR;
        if (!mbar_wait(&rempty[r], ((it / ZNR) & 1) ^ 1, &abort_s, P.status)) break;
        const long long sg = W.s0 + st_;
        const float2* src = P.rho + (size_t)sg * P.gpad * ZK;
        const uint32_t dst = rbase + r * ZR_STAGE;
        mbar_expect_tx(&rfull[r], bi + bj + ZK * 16);
        bulk_g2s(dst, src + (size_t)W.I * ZG * ZK, bi, &rfull[r]);
        if (bj) bulk_g2s(dst + ZRB, src + (size_t)W.J * ZG * ZK, bj, &rfull[r]);
        bulk_g2s(dst + ZR_PW, P.pw + sg * ZK, ZK * 16, &rfull[r]);
      }
      // wait (bounded) for the copies that may still be in flight (it: stages issued)
      for (uint32_t j = (it > (uint32_t)ZNR ? it - ZNR : 0u); j < it; ++j)
        mbar_drain(&rfull[j % ZNR], (j / ZNR) & 1, P.status);
    }
  } else if (warp == ZW_MMA) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = (1u << 4) | ((BF ? 1u : 0u) << 7) | ((BF ? 1u : 0u) << 10) | (1u << 15) |
                           (1u << 16) | ((uint32_t)(ZM >> 3) << 17) | ((uint32_t)(ZM >> 4) << 24);
    bool ok = true;
    uint32_t it = 0, pc = 0;
    for (int p0 = 0; p0 < nst && ok; p0 += ZPERIOD, ++pc) {
      const int buf = pc & 1, p1 = min(nst, p0 + ZPERIOD);
      if (lane == 0) ok = mbar_wait(&acc_empty[buf], ((pc >> 1) & 1) ^ 1, &abort_s, P.status);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc_fence_after();
      const uint32_t d = tmem + buf * ZM;
      for (int st_ = p0; st_ < p1; ++st_, ++it) {
        const int s = it % ZNS;
        if (lane == 0) ok = mbar_wait(&full[s], (it / ZNS) & 1, &abort_s, P.status);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        tc_fence_after();
        if (lane == 0) {
          const uint32_t sa = base + s * ZSTAGE;
#pragma unroll
          for (int kk = 0; kk < ZK / 16; ++kk) {
            const uint64_t aH = sdesc(sa + kk * 2 * ZSBO, 1024, ZSBO);
            const uint64_t aL = sdesc(sa + ZA_BYTES + kk * 2 * ZSBO, 1024, ZSBO);
            const uint64_t bH = sdesc(sa + 2 * ZA_BYTES + kk * 2 * ZSBO, 1024, ZSBO);
            const uint64_t bL = sdesc(sa + 3 * ZA_BYTES + kk * 2 * ZSBO, 1024, ZSBO);
            mma1(d, aH, bH, idesc, (st_ > p0 || kk > 0) ? 1u : 0u);
            mma1(d, aH, bL, idesc, 1u);
            mma1(d, aL, bH, idesc, 1u);
          }
          mma1_commit(&empty[s]);
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) mma1_commit(&acc_full[buf]);
      __syncwarp();
    }
    if (lane == 0) {
      mma1_commit(&final_bar);
      mbar_drain(&final_bar, 0, P.status);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: accumulator rows into this CTA's FP64 partial sums --------
    const int q = warp & 3;              // tensor-memory lane quadrant of this warp
    const int m = q * 32 + lane;         // row (G, Re|Im)
    double* part = P.part + (size_t)blockIdx.x * ZM * ZM + m;
    uint32_t pc = 0;
    for (int p0 = 0; p0 < nst; p0 += ZPERIOD, ++pc) {
      const int buf = pc & 1;
      bool ok = true;
      if (lane == 0) ok = mbar_wait(&acc_full[buf], (pc >> 1) & 1, &abort_s, P.status);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc_fence_after();
#pragma unroll 1
      for (int c = 0; c < ZM / 16; ++c) {
        uint32_t v[16];
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + buf * ZM + c * 16;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        double* pp = part + (size_t)(c * 16) * ZM;
        double old[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) old[j] = pp[(size_t)j * ZM];
#pragma unroll
        for (int j = 0; j < 16; ++j) pp[(size_t)j * ZM] = old[j] + (double)__uint_as_float(v[j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == ZW_MMA)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * ZM));
}

// chi0(G, G') of tile t = (I, J) from the partial sums of its CTAs (b = t, t + ntile, ...):
// chi0 = scale ((C_rr - C_ii) + i (C_ri + C_ir)), C_ab at row 2 g + a, column 2 g' + b.
__global__ void chi0_zero_tc_reduce(const double* __restrict__ part, int grid, int ntile, int rt,
                                    int nG, double scale, double2* __restrict__ out) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)ntile * ZG * ZG) return;
  const int t = (int)(idx / (ZG * ZG)), gp = (int)((idx / ZG) % ZG), g = (int)(idx % ZG);
  const int G = (t / rt) * ZG + g, Gp = (t % rt) * ZG + gp;
  if (G >= nG || Gp >= nG) return;
  double rr = 0.0, ir = 0.0, ri = 0.0, ii = 0.0;
  for (int b = t; b < grid; b += ntile) {
    const double* pb = part + (size_t)b * ZM * ZM;
    const double2 x = *reinterpret_cast<const double2*>(pb + (size_t)(2 * gp) * ZM + 2 * g);
    const double2 y = *reinterpret_cast<const double2*>(pb + (size_t)(2 * gp + 1) * ZM + 2 * g);
    rr += x.x;
    ir += x.y;
    ri += y.x;
    ii += y.y;
  }
  out[(size_t)G * nG + Gp] = make_double2(scale * (rr - ii), scale * (ri + ir));
}

}  // namespace

// The w = 0 column of every eta on the tensor cores; *done = false (nothing launched) when the
// tiles outnumber the SMs, for the caller's SIMT kernel.
lrt_status launch_zero_tc(const lrt_ctx* c, QData& q, const void* rho, float sB, cudaStream_t s,
                          bool* done) {
  *done = false;
  const int nG = q.nG;
  const int rt = (nG + ZG - 1) / ZG, ntile = rt * rt;
  int dev = 0, nsm = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (ntile > nsm) return LRT_OK;
  const int grid = nsm;
  const size_t part_bytes = (size_t)grid * ZM * ZM * sizeof(double);
  lrt_ctx* cc = const_cast<lrt_ctx*>(c);
  if (cc->dw.zt_bytes < part_bytes) {
    cudaFree(cc->dw.zt_part);
    cc->dw.zt_part = nullptr;
    cc->dw.zt_bytes = 0;
    LRT_CUDA(cudaMalloc(&cc->dw.zt_part, part_bytes));
    cc->dw.zt_bytes = part_bytes;
  }
  const bool bf = c->precision == LRT_PREC_BF16X3;
  auto kern = bf ? chi0_zero_tc_kernel<true> : chi0_zero_tc_kernel<false>;
  // raised once per device and form (repeated calls and graph captures make no attribute call)
  static bool attr_set[64][2] = {};
  if (dev < 0 || dev >= 64 || !attr_set[dev][bf]) {
    LRT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ZSMEM));
    if (dev >= 0 && dev < 64) attr_set[dev][bf] = true;
  }
  const double r = split_rho_scale(c->precision);
  const double scale = 2.0 / (c->nk * c->volume) / (r * (double)sB);
  const long long mat = (long long)nG * nG;
  ZParams P;
  P.rho = (const float2*)rho;
  P.pw = q.sp.pw;
  P.part = cc->dw.zt_part;
  P.status = c->dw.status;
  P.nstage = (c->np + ZK - 1) / ZK;
  P.gpad = c->rho_gpad;
  P.ntile = ntile;
  P.rt = rt;
  P.inv_r = (float)(1.0 / r);
  const long long nred = (long long)ntile * ZG * ZG;
  for (int e = 0; e < c->neta; ++e) {
    P.eta = (float)c->etas[e];
    LRT_CUDA(cudaMemsetAsync(P.part, 0, part_bytes, s));
    kern<<<grid, ZTHREADS, ZSMEM, s>>>(P);
    count_launch(c);
    LRT_CUDA(cudaGetLastError());
    double2* out = q.chi0 + ((size_t)c->hcol + (size_t)e * c->nwi) * mat;
    chi0_zero_tc_reduce<<<(unsigned)((nred + 255) / 256), 256, 0, s>>>(P.part, grid, ntile, rt, nG, scale, out);
    count_launch(c);
    LRT_CUDA(cudaGetLastError());
  }
  *done = true;
  return LRT_OK;
}

}  // namespace lrt
