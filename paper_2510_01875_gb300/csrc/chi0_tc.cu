// Split-precision Adler-Wiser chi0 on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The contraction chi0_GG'(w) = pref sum_p rho_p(G) rho_p*(G') w_p(w) is run as one real GEMM
//   C[r][c] = sum_p A[r][p] B[p][c]
// with Hermitian-split rows r = (G <= G', Re|Im of P_p = rho_p(G) rho_p*(G')) and columns
// c = (w, Re|Im of w_p(w) = df_p / (w + Delta_p + i eta)).  From RR, RI, IR, II of a row pair
// and a column pair, chi0(G,G') = (RR - II) + i(RI + IR) and chi0(G',G) = (RR + II) + i(RI - IR).
//
// Both operands are generated inside the kernel and never stored in global memory.  Per
// 32-pair stage:
//  - a loader warp copies the stage's rho rows (blocked layout rho[p/32][G][p%32]: one 2 KB
//    bulk copy per 8-G block the row tile touches) and the 32 (Delta_hi, Delta_lo, df) into a
//    shared-memory ring with cp.async.bulk, completion counted in bytes on an mbarrier;
//  - 16 producer warps form P (8 warps, 256 rows) and w (8 warps, 256 columns) in FP32, with
//    w + Delta carried as (hi, lo) floats so the sum keeps FP64-level accuracy when it
//    cancels, split every value v into v_hi = round16(v) and v_lo = round16(v - v_hi) (FP16
//    with power-of-two scales, or BF16), and write the tiles MN-major with the 128-byte
//    swizzle (each lane owns one pair = one K index and stores 16-byte chunks of 8 rows or
//    columns);
//  - one thread issues tcgen05.mma kind::f16, M = 128, N = 256, K = 16, for
//    A_hi B_hi + A_hi B_lo + A_lo B_hi into two FP32 accumulators in tensor memory (two row
//    tiles share each B tile: 256 x 256 outputs per CTA);
//  - every `flush` stages four epilogue warps read the accumulators (tcgen05.ld) and add them
//    into a per-CTA double-float (FP32 hi + lo, two-sum) slab in global memory; at the end of
//    a unit the slab is added into the FP64 sums C.
// Units of work are (row super-tile, column tile, pair range), handed out round-robin to one
// CTA per SM.  Every wait on an mbarrier is bounded; on expiry the kernel sets bit 2 of the
// status word, stops issuing work, waits (bounded) for its own copies and MMAs and frees its
// tensor memory before returning.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "lrt_internal.h"

namespace lrt {
namespace {

constexpr int TM = 128;            // rows per accumulator (64 row pairs)
constexpr int NACC = 2;            // accumulators (row tiles) per CTA
constexpr int TN = 256;            // columns per tile (128 frequencies)
constexpr int KS = 32;             // pairs (K) per pipeline stage
constexpr int NS = 2;              // operand (A/B) stages
constexpr int NSR = 6;             // prefetch stages of rho blocks and pair weights
constexpr int GBLK = 8;            // G per block of the blocked rho layout
constexpr int MAXBLK = 6;          // G blocks one row super-tile may touch
constexpr int RROWS = MAXBLK * GBLK;
constexpr int NPROD = 16;          // producer warps 0..15: 0..7 build A, 8..15 build B
constexpr int WMMA = 16;           // MMA warp
constexpr int WLOAD = 21;          // loader warp
constexpr int NTHREADS = 22 * 32;  // + epilogue warps 17..20 (one per TMEM lane quadrant)
constexpr int CHUNKS = 4;          // 16-byte chunks (8 rows or columns) per producer warp
constexpr int A_BYTES = TM * KS * 2;                 // 8 KB per 16-bit row tile
constexpr int B_BYTES = TN * KS * 2;                 // 16 KB
constexpr int STAGE_BYTES = NACC * 2 * A_BYTES + 2 * B_BYTES;   // 64 KB
constexpr int A_SBO = (TM / 64) * 1024;              // bytes between 8-pair groups of A
constexpr int B_SBO = (TN / 64) * 1024;
constexpr int RBLK_BYTES = GBLK * KS * 8;            // one G block of one stage: 2 KB
constexpr int R_STAGE = RROWS * KS * 8 + KS * 16;    // rho rows + 32 float4 pair weights
constexpr unsigned long long kTimeoutNs = 2000000000ull;
constexpr int kFlushStages = 128;  // FP32 accumulation period: 128 stages = 4096 pairs

struct Params {
  const float2* rho;          // blocked [ld/32][gpad][32]
  const float4* pw;           // [np rounded up to 32] {Delta_hi, Delta_lo, df, 0}
  const int2* rowtab;         // [n_st * 128] local (G, G') indices per row pair, -1 padding
  const int* blk;             // [n_st * MAXBLK] G blocks of the super-tile, -1 padding
  const float2* wtab;         // [n_n * 128] frequency hi/lo per column pair
  double* C;                  // [n_n * TN][ldr] FP64 sums, column-major
  float2* slab;               // [gridDim.x][TN][NACC * TM] per-CTA (hi, lo), column-major
  int* status;
  long long np;
  long long ldr;              // = n_st * NACC * TM
  int gpad;
  int rows_valid;             // 2 * row pairs
  int cols_valid;             // 2 * nwi
  int n_st, n_n, n_split;
  long long k_per_split;      // multiple of KS
  int flush;                  // stages per accumulator period
  float eta, sA, sB;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(n));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// try_wait with a suspend-time hint: the warp sleeps in hardware until the phase completes or
// about `hint_ns` passes, instead of spinning on the issue slots.
__device__ __forceinline__ bool mbar_try_sleep(uint64_t* b, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when this CTA is aborting or the wait ran out (then it starts the abort).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag,
                                          int* status) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = gtime();
  while (!mbar_try_sleep(b, parity, 20000u)) {
    if (*abort_flag) return false;
    if (gtime() - t0 > kTimeoutNs) {
      *abort_flag = 1;
      atomicOr(status, 2);
      return false;
    }
  }
  return true;
}
// Bounded wait used while draining: ignores the abort flag.
__device__ __forceinline__ void mbar_drain(uint64_t* b, uint32_t parity, int* status) {
  const unsigned long long t0 = gtime();
  while (!mbar_try_sleep(b, parity, 20000u)) {
    if (gtime() - t0 > kTimeoutNs) {
      atomicOr(status, 2);
      return;
    }
  }
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_u32(b)),
               "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared, completion counted in bytes on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: start >> 4, LBO >> 4 at bit 16, SBO >> 4 at bit 32,
// version 1 at bit 46, 128-byte swizzle (2) at bits 61-63.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(b))
      : "memory");
}

// Offset of the 16-byte chunk holding MN elements [8c, 8c+8) of K index k in an MN-major,
// 128-byte-swizzled tile: [k/8][mn/64][k%8][64 elements], chunk (mn%64)/8 XOR k%8.
__device__ __forceinline__ uint32_t mn_chunk(int k, int c, int sbo) {
  return (uint32_t)((k >> 3) * sbo + (c >> 3) * 1024 + (k & 7) * 128 + (((c & 7) ^ (k & 7)) << 4));
}

template <bool BF>
struct Pack;
template <>
struct Pack<false> {
  // 8 floats -> hi and lo as 8 x f16 each
  __device__ __forceinline__ static void split(const float* v, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2 a = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
      float2 af = __half22float2(a);
      __half2 b = __floats2half2_rn(v[2 * i] - af.x, v[2 * i + 1] - af.y);
      h[i] = *reinterpret_cast<uint32_t*>(&a);
      l[i] = *reinterpret_cast<uint32_t*>(&b);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
  }
};
template <>
struct Pack<true> {
  __device__ __forceinline__ static void split(const float* v, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __nv_bfloat162 a = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      float2 af = __bfloat1622float2(a);
      __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * i] - af.x, v[2 * i + 1] - af.y);
      h[i] = *reinterpret_cast<uint32_t*>(&a);
      l[i] = *reinterpret_cast<uint32_t*>(&b);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
  }
};

// No memory clobber: the operand tiles are read only by the tensor cores after the
// fence.proxy.async + mbarrier arrive that follow (volatile asm keeps that order), so the
// compiler may hoist the next chunk's loads above these stores.
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w));
}

struct Unit {
  int st, nt;
  long long kb, ke;
};
__device__ __forceinline__ Unit unit_of(const Params& P, int u) {
  Unit U;
  int tile = u / P.n_split, ks = u % P.n_split;
  U.st = tile / P.n_n;
  U.nt = tile % P.n_n;
  U.kb = (long long)ks * P.k_per_split;
  U.ke = min(P.np, U.kb + P.k_per_split);
  return U;
}

template <bool BF>
__global__ void __launch_bounds__(NTHREADS, 1) chi0_tc_kernel(Params P) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[NS], empty[NS], acc_full, acc_empty, final_bar;
  __shared__ __align__(8) uint64_t rfull[NSR], rempty[NSR];
  __shared__ uint32_t tmem_base_s;
  __shared__ int2 rowtab_s[NACC * 64];
  __shared__ int blk_s[MAXBLK];
  __shared__ int nblk_s;
  __shared__ float2 wtab_s[128];
  __shared__ volatile int abort_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t* base_gen = smem_raw + (base - smem_u32(smem_raw));
  const uint32_t rbase = base + NS * STAGE_BYTES;          // prefetch ring
  const uint8_t* rbase_gen = base_gen + NS * STAGE_BYTES;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], NPROD);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < NSR; ++s) {
      mbar_init(&rfull[s], 1);
      mbar_init(&rempty[s], NPROD);
    }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, 4);
    mbar_init(&final_bar, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == WMMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(NACC * TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  const int nunits = P.n_st * P.n_n * P.n_split;
  const uint32_t idesc = (1u << 4) | ((BF ? 1u : 0u) << 7) | ((BF ? 1u : 0u) << 10) | (1u << 15) |
                         (1u << 16) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

  uint32_t it = 0;   // stage counter (producers, loader, MMA)
  uint32_t pc = 0;   // accumulator period counter (MMA and epilogue)
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const Unit U = unit_of(P, u);
    // per-unit tables (row pairs and G blocks of the super-tile, frequencies of the column tile)
    __syncthreads();
    if (threadIdx.x < NACC * 64) rowtab_s[threadIdx.x] = P.rowtab[U.st * NACC * 64 + threadIdx.x];
    if (threadIdx.x < 128) wtab_s[threadIdx.x] = P.wtab[U.nt * 128 + threadIdx.x];
    if (threadIdx.x < MAXBLK) blk_s[threadIdx.x] = P.blk[U.st * MAXBLK + threadIdx.x];
    if (threadIdx.x == 0) {
      int n = 0;
      while (n < MAXBLK && P.blk[U.st * MAXBLK + n] >= 0) ++n;
      nblk_s = n;
    }
    __syncthreads();
    if (abort_s) break;
    const long long nstage = (U.ke - U.kb + KS - 1) / KS;
    const long long nper = (nstage + P.flush - 1) / P.flush;

    if (warp < NPROD) {
      // ---------------- producers ----------------
      for (long long st = 0; st < nstage; ++st, ++it) {
        const int s = it % NS, sr = it % NSR;
        // every lane waits; the vote keeps the warp together if one lane's wait gives up
        if (!__all_sync(0xffffffffu, mbar_wait(&rfull[sr], (it / NSR) & 1, &abort_s, P.status)))
          break;
        if (!__all_sync(0xffffffffu, mbar_wait(&empty[s], ((it / NS) & 1) ^ 1, &abort_s, P.status)))
          break;
        const long long p = U.kb + st * KS + lane;
        const bool valid = p < U.ke;
        const float2* rrow = reinterpret_cast<const float2*>(rbase_gen + sr * R_STAGE) + lane;
        const float4* rpw =
            reinterpret_cast<const float4*>(rbase_gen + sr * R_STAGE + RROWS * KS * 8);
        const float4 pw = valid ? rpw[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t sst = base + s * STAGE_BYTES;
        if (warp < 8) {
#pragma unroll
          for (int cc = 0; cc < CHUNKS; ++cc) {
            const int c = CHUNKS * warp + cc;        // 0..31: row tile c/16, chunk c%16
            const int a = c >> 4, cl = c & 15;
            float v[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int2 g = rowtab_s[a * 64 + 4 * cl + i];
              float pr = 0.f, pi = 0.f;
              if (valid && g.x >= 0) {
                const float2 x = rrow[g.x * KS];
                const float2 y = rrow[g.y * KS];
                pr = (x.x * y.x + x.y * y.y) * P.sA;
                pi = (x.y * y.x - x.x * y.y) * P.sA;
              }
              v[2 * i] = pr;
              v[2 * i + 1] = pi;
            }
            uint4 hi, lo;
            Pack<BF>::split(v, hi, lo);
            const uint32_t ahi = sst + a * 2 * A_BYTES;
            st_shared_v4(ahi + mn_chunk(lane, cl, A_SBO), hi);
            st_shared_v4(ahi + A_BYTES + mn_chunk(lane, cl, A_SBO), lo);
          }
        } else {
          const float dfs = pw.z * P.sB;
#pragma unroll
          for (int cc = 0; cc < CHUNKS; ++cc) {
            const int cb = CHUNKS * (warp - 8) + cc;  // 0..31: columns 8 cb ..
            float v[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float2 w = wtab_s[4 * cb + i];
              const float x = (w.x + pw.x) + (w.y + pw.y);
              const float d = fmaf(x, x, P.eta * P.eta);
              const float sc = __fdividef(dfs, d);
              v[2 * i] = sc * x;
              v[2 * i + 1] = -sc * P.eta;
            }
            uint4 hi, lo;
            Pack<BF>::split(v, hi, lo);
            const uint32_t bhi = sst + NACC * 2 * A_BYTES;
            st_shared_v4(bhi + mn_chunk(lane, cb, B_SBO), hi);
            st_shared_v4(bhi + B_BYTES + mn_chunk(lane, cb, B_SBO), lo);
          }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&full[s]);
          mbar_arrive(&rempty[sr]);
        }
      }
    } else if (warp == WLOAD) {
      // ---------------- loader: rho blocks and pair weights of each stage ----------------
      if (lane == 0) {
        const int nb = nblk_s;
        const uint32_t bytes = (uint32_t)(nb * RBLK_BYTES + KS * 16);
        for (long long st = 0; st < nstage; ++st, ++it) {
          const int sr = it % NSR;
          if (!mbar_wait(&rempty[sr], ((it / NSR) & 1) ^ 1, &abort_s, P.status)) break;
          const long long p0 = U.kb + st * KS;
          mbar_expect_tx(&rfull[sr], bytes);
          const uint32_t dst = rbase + sr * R_STAGE;
          const float2* src = P.rho + (size_t)(p0 >> 5) * P.gpad * KS;
          for (int i = 0; i < nb; ++i)
            bulk_g2s(dst + i * RBLK_BYTES, src + (size_t)blk_s[i] * GBLK * KS, RBLK_BYTES, &rfull[sr]);
          bulk_g2s(dst + RROWS * KS * 8, P.pw + p0, KS * 16, &rfull[sr]);
        }
      }
      it = __shfl_sync(0xffffffffu, it, 0);
    } else if (warp == WMMA) {
      // ---------------- MMA issuer ----------------
      for (long long per = 0; per < nper; ++per, ++pc) {
        bool ok = true;
        if (lane == 0) ok = mbar_wait(&acc_empty, (pc & 1) ^ 1, &abort_s, P.status);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        tc_fence_after();
        const long long s0 = per * P.flush, s1 = min(nstage, s0 + P.flush);
        for (long long st = s0; st < s1; ++st, ++it) {
          const int s = it % NS;
          if (lane == 0) ok = mbar_wait(&full[s], (it / NS) & 1, &abort_s, P.status);
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (!ok) break;
          tc_fence_after();
          if (lane == 0) {
            const uint32_t sst = base + s * STAGE_BYTES;
            const uint32_t bH = sst + NACC * 2 * A_BYTES, bL = bH + B_BYTES;
#pragma unroll
            for (int kk = 0; kk < KS / 16; ++kk) {
              const uint64_t dBh = sdesc(bH + kk * 2 * B_SBO, 1024, B_SBO);
              const uint64_t dBl = sdesc(bL + kk * 2 * B_SBO, 1024, B_SBO);
#pragma unroll
              for (int a = 0; a < NACC; ++a) {
                const uint32_t aH = sst + a * 2 * A_BYTES, aL = aH + A_BYTES;
                const uint64_t dAh = sdesc(aH + kk * 2 * A_SBO, 1024, A_SBO);
                const uint64_t dAl = sdesc(aL + kk * 2 * A_SBO, 1024, A_SBO);
                const uint32_t d = tmem + a * TN;
                mma(d, dAh, dBh, idesc, (st > s0 || kk > 0) ? 1u : 0u);
                mma(d, dAh, dBl, idesc, 1u);
                mma(d, dAl, dBh, idesc, 1u);
              }
            }
            mma_commit(&empty[s]);
          }
          __syncwarp();
        }
        if (!ok) break;
        if (lane == 0) mma_commit(&acc_full);
        __syncwarp();
      }
    } else {
      // ---------------- epilogue ----------------
      // The unit's sums live in a per-CTA column-major slab of (hi, lo) float pairs
      // (double-float, two-sum accumulation; a warp touches 32 consecutive rows per column)
      // and are added into the FP64 sums C when the unit's pair range is done.
      const int q = warp & 3;            // tensor-memory lane quadrant of this warp
      float2* slab = P.slab + (size_t)blockIdx.x * TN * (NACC * TM);
      bool unit_ok = true;
      for (long long per = 0; per < nper; ++per, ++pc) {
        bool ok = true;
        if (lane == 0) ok = mbar_wait(&acc_full, pc & 1, &abort_s, P.status);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          unit_ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll 1
        for (int a = 0; a < NACC; ++a) {
          const int row = a * TM + q * 32 + lane;
#pragma unroll 1
          for (int c = 0; c < TN / 16; ++c) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + a * TN + c * 16;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
                "%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float2* col = slab + (size_t)(c * 16) * (NACC * TM) + row;
            if (per == 0) {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                col[(size_t)j * (NACC * TM)] = make_float2(__uint_as_float(r[j]), 0.f);
            } else {
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                float2 h = col[(size_t)j * (NACC * TM)];
                const float v = __uint_as_float(r[j]);
                const float s = h.x + v;                 // two-sum of h.x + v
                const float bp = s - h.x;
                const float err = (h.x - (s - bp)) + (v - bp);
                col[(size_t)j * (NACC * TM)] = make_float2(s, h.y + err);
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty);
      }
      if (unit_ok) {
        const int col0 = U.nt * TN;
        for (int a = 0; a < NACC; ++a) {
          const int row = a * TM + q * 32 + lane;
          const long long grow = (long long)U.st * (NACC * TM) + row;
          if (grow >= P.rows_valid) continue;
          for (int j = 0; j < TN && col0 + j < P.cols_valid; ++j) {
            const float2 h = slab[(size_t)j * (NACC * TM) + row];
            atomicAdd(P.C + (size_t)(col0 + j) * P.ldr + grow, (double)h.x + (double)h.y);
          }
        }
      }
    }
    // keep every role on the same unit; an abort stops all of them
    __syncthreads();
  }
  // drain: the loader waits (bounded) for its last bulk copies, the MMA warp for this CTA's
  // MMAs, before the shared and tensor memory go away
  if (warp == WLOAD && lane == 0) {
    for (uint32_t j = (it > (uint32_t)NSR ? it - NSR : 0u); j < it; ++j)
      mbar_drain(&rfull[j % NSR], (j / NSR) & 1, P.status);
  }
  if (warp == WMMA) {
    if (lane == 0) {
      mma_commit(&final_bar);
      mbar_drain(&final_bar, 0, P.status);
    }
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == WMMA)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NACC * TN));
}

// chi0[w][G][G'] from the FP64 sums (C column-major: C[col * ldr + row])
__global__ void chi0_unpack(const double* __restrict__ C, long long ldr,
                            const int* __restrict__ rp_of, int nG, int nwi, double scale,
                            double2* __restrict__ chi0) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long total = (long long)nwi * nG * nG;
  if (t >= total) return;
  int Gp = (int)(t % nG);
  int G = (int)((t / nG) % nG);
  int w = (int)(t / ((long long)nG * nG));
  int rp = rp_of[G * nG + Gp];
  const double* cre = C + (long long)(2 * w) * ldr;       // column Re w
  const double* cim = C + (long long)(2 * w + 1) * ldr;   // column Im w
  double RR = cre[2 * rp], IR = cre[2 * rp + 1], RI = cim[2 * rp], II = cim[2 * rp + 1];
  double2 v;
  if (G <= Gp)
    v = make_double2(RR - II, RI + IR);
  else
    v = make_double2(RR + II, RI - IR);
  chi0[t] = make_double2(scale * v.x, scale * v.y);
}

// {Delta_hi, Delta_lo, df, 0} per pair (Delta split so that w + Delta keeps FP64-level
// accuracy when it cancels in FP32); df carries the band weights.
__global__ void pair_weights_split(const double* __restrict__ eps, const double* __restrict__ occ,
                                   const double* __restrict__ wgt, int nk, int nb,
                                   float4* __restrict__ pw) {
  long long np = (long long)nk * nb * nb;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    int m = (int)(p % nb);
    long long kn = p / nb;
    int k = (int)(kn / nb);
    size_t ikq = (size_t)(nk + k) * nb + m;
    double d = eps[kn] - eps[ikq];
    float dh = (float)d;
    pw[p] = make_float4(dh, (float)(d - (double)dh),
                        (float)(wgt[kn] * wgt[ikq] * (occ[kn] - occ[ikq])), 0.f);
  }
}

}  // namespace

lrt_status launch_chi0_split(const lrt_ctx* c, QData& q, cudaStream_t s) {
  const int nG = q.nG;
  if (c->np <= 0) {
    set_error("no pairs to contract");
    return LRT_EINVAL;
  }
  if (c->rho_gpad < (nG + GBLK - 1) / GBLK * GBLK) {
    set_error("pair densities are not in the blocked layout");
    return LRT_ESTATE;
  }
  // row pairs (G <= G') in 8 x 8 blocks so that a row tile touches few G blocks
  std::vector<int2> pairs;
  const int nblk = (nG + GBLK - 1) / GBLK;
  for (int I = 0; I < nblk; ++I)
    for (int J = I; J < nblk; ++J)
      for (int a = I * GBLK; a < std::min(nG, I * GBLK + GBLK); ++a)
        for (int b = J * GBLK; b < std::min(nG, J * GBLK + GBLK); ++b)
          if (I < J || a <= b) pairs.push_back(make_int2(a, b));
  const int npairs = (int)pairs.size();
  const int per_st = NACC * 64;                       // row pairs per super-tile
  const int n_st = (npairs + per_st - 1) / per_st;
  std::vector<int2> rowtab((size_t)n_st * per_st, make_int2(-1, -1));
  std::vector<int> blk((size_t)n_st * MAXBLK, -1);
  std::vector<int> rp_of((size_t)nG * nG);
  for (int i = 0; i < npairs; ++i) {
    rp_of[pairs[i].x * nG + pairs[i].y] = i;
    rp_of[pairs[i].y * nG + pairs[i].x] = i;
  }
  for (int t = 0; t < n_st; ++t) {
    int* bl = &blk[(size_t)t * MAXBLK];
    int n = 0;
    auto slot = [&](int G) {
      const int b = G / GBLK;
      for (int i = 0; i < n; ++i)
        if (bl[i] == b) return i * GBLK + G % GBLK;
      if (n == MAXBLK) return -1;
      bl[n] = b;
      return (n++) * GBLK + G % GBLK;
    };
    for (int r = 0; r < per_st && t * per_st + r < npairs; ++r) {
      const int2 pr = pairs[t * per_st + r];
      const int la = slot(pr.x), lb = slot(pr.y);
      if (la < 0 || lb < 0) {
        set_error("a row super-tile touches more than 6 G blocks");
        return LRT_EUNSUPPORTED;
      }
      rowtab[(size_t)t * per_st + r] = make_int2(la, lb);
    }
  }
  const int ncols = 2 * c->nwi;
  const int n_n = (ncols + TN - 1) / TN;
  std::vector<float2> wtab((size_t)n_n * 128, make_float2(0.f, 0.f));
  for (int j = 0; j < c->nwi; ++j) {
    float h = (float)c->freqs[j];
    wtab[j] = make_float2(h, (float)(c->freqs[j] - (double)h));
  }
  const bool bf = c->precision == LRT_PREC_BF16X3;
  const float sA = bf ? 1.0f : 16384.0f;
  float sB = 1.0f;
  if (!bf) sB = std::ldexp(1.0f, (int)std::floor(std::log2(16384.0 * c->eta)));
  const int ldc = n_n * TN;

  int dev = 0, nsm = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const long long tiles = (long long)n_st * n_n;
  // pair splits: at least 4 units per SM, chosen to fill the last round
  long long best_split = 1;
  double best_eff = 0.0;
  const long long max_split = std::max<long long>(1, c->np / (KS * 64));
  for (long long sp = std::max<long long>(1, (4LL * nsm + tiles - 1) / tiles);
       sp <= 8LL * nsm / std::max<long long>(1, tiles) + 8 && sp <= max_split; ++sp) {
    long long units = tiles * sp;
    double eff = (double)units / (double)(((units + nsm - 1) / nsm) * nsm);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best_split = sp;
    }
  }
  long long kps = (c->np + best_split - 1) / best_split;
  kps = (kps + KS - 1) / KS * KS;
  const int n_split = (int)((c->np + kps - 1) / kps);

  // device buffers: C (column-major FP64 sums) then the per-CTA slabs
  const long long ldr = (long long)n_st * NACC * TM;
  const long long units = tiles * n_split;
  const int grid = (int)std::min<long long>(nsm, units);
  const size_t c_bytes = (size_t)ldr * ldc * sizeof(double);
  const size_t need = c_bytes + (size_t)grid * TN * NACC * TM * sizeof(float2);
  DeviceWork& dw = const_cast<DeviceWork&>(c->dw);
  if (dw.scratch_bytes < need) {
    cudaFree(dw.scratch);
    dw.scratch = nullptr;
    dw.scratch_bytes = 0;
    LRT_CUDA(cudaMalloc(&dw.scratch, need));
    dw.scratch_bytes = need;
  }
  int2* d_rowtab = nullptr;
  int* d_blk = nullptr;
  int* d_rp = nullptr;
  float2* d_wtab = nullptr;
  float4* d_pw = nullptr;
  // pair weights padded to whole 32-pair stages (the bulk copies read full stages)
  const size_t npw_pad = (size_t)((c->np + KS - 1) / KS * KS);
  LRT_CUDA(cudaMallocAsync(&d_rowtab, rowtab.size() * sizeof(int2), s));
  LRT_CUDA(cudaMallocAsync(&d_blk, blk.size() * sizeof(int), s));
  LRT_CUDA(cudaMallocAsync(&d_rp, rp_of.size() * sizeof(int), s));
  LRT_CUDA(cudaMallocAsync(&d_wtab, wtab.size() * sizeof(float2), s));
  LRT_CUDA(cudaMallocAsync(&d_pw, npw_pad * sizeof(float4), s));
  LRT_CUDA(cudaMemsetAsync(d_pw, 0, npw_pad * sizeof(float4), s));
  LRT_CUDA(cudaMemcpyAsync(d_rowtab, rowtab.data(), rowtab.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
  LRT_CUDA(cudaMemcpyAsync(d_blk, blk.data(), blk.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  LRT_CUDA(cudaMemcpyAsync(d_rp, rp_of.data(), rp_of.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  LRT_CUDA(cudaMemcpyAsync(d_wtab, wtab.data(), wtab.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
  pair_weights_split<<<4 * nsm, 256, 0, s>>>(q.eps, q.occ, q.wgt, c->nk, c->nb, d_pw);
  LRT_CUDA(cudaGetLastError());
  LRT_CUDA(cudaMemsetAsync(dw.scratch, 0, c_bytes, s));

  Params P;
  P.rho = (const float2*)dw.rho;
  P.pw = d_pw;
  P.rowtab = d_rowtab;
  P.blk = d_blk;
  P.wtab = d_wtab;
  P.C = dw.scratch;
  P.slab = reinterpret_cast<float2*>(dw.scratch + (size_t)ldr * ldc);
  P.status = dw.status;
  P.np = c->np;
  P.ldr = ldr;
  P.gpad = c->rho_gpad;
  P.rows_valid = 2 * npairs;
  P.cols_valid = ncols;
  P.n_st = n_st;
  P.n_n = n_n;
  P.n_split = n_split;
  P.k_per_split = kps;
  P.flush = kFlushStages;
  P.eta = (float)c->eta;
  P.sA = sA;
  P.sB = sB;
  const size_t smem = (size_t)NS * STAGE_BYTES + (size_t)NSR * R_STAGE + 1024;
  if (bf)
    LRT_CUDA(cudaFuncSetAttribute(chi0_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  else
    LRT_CUDA(cudaFuncSetAttribute(chi0_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    TimedLaunch tl(c, &c->ev_chi0, s);
    if (bf)
      chi0_tc_kernel<true><<<grid, NTHREADS, smem, s>>>(P);
    else
      chi0_tc_kernel<false><<<grid, NTHREADS, smem, s>>>(P);
  }
  count_launch(c, 2);   // pair_weights_split + the contraction
  if (c->profiling) c->timed_cmac += (double)nG * nG * c->nw * (double)c->np;
  LRT_CUDA(cudaGetLastError());
  const double scale = 2.0 / (c->nk * c->volume) / ((double)sA * (double)sB);
  long long total = (long long)c->nwi * nG * nG;
  chi0_unpack<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(dw.scratch, ldr, d_rp, nG, c->nwi, scale,
                                                             q.chi0);
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  LRT_CUDA(cudaFreeAsync(d_rowtab, s));
  LRT_CUDA(cudaFreeAsync(d_blk, s));
  LRT_CUDA(cudaFreeAsync(d_rp, s));
  LRT_CUDA(cudaFreeAsync(d_wtab, s));
  LRT_CUDA(cudaFreeAsync(d_pw, s));
  return LRT_OK;
}

}  // namespace lrt
