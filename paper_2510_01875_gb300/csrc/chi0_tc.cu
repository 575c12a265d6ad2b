// Split-precision Adler-Wiser chi0 on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The contraction chi0_GG'(w) = pref sum_p rho_p(G) rho_p*(G') w_p(w) is run as one real GEMM
//   C[r][c] = sum_p A[r][p] B[p][c]
// with Hermitian-split rows r = (G <= G', Re|Im of P_p = rho_p(G) rho_p*(G')) and columns
// c = (w, Re|Im of w_p(w) = df_p / (w + Delta_p + i eta)).  From RR, RI, IR, II of a row pair
// and a column pair, chi0(G,G') = (RR - II) + i(RI + IR) and chi0(G',G) = (RR + II) + i(RI - IR).
//
// Both operands are generated inside the kernel and never stored in global memory.  A cluster
// of two CTAs (one per SM) works as a pair with tcgen05.mma.cta_group::2 (M = 256, N = 256,
// K = 16): each CTA builds its own 2 x 128 rows of A and half (128 columns) of the shared B
// tile, and each CTA's tensor memory holds its rows of the two 256 x 256 accumulators.  Per
// 32-pair stage:
//  - a loader warp copies the stage's rho rows (blocked layout rho[p/32][G][p%32]: one 2 KB
//    bulk copy per 8-G block the CTA's rows touch) and the 32 (Delta_hi, Delta_lo, df) into a
//    shared-memory ring with cp.async.bulk, completion counted in bytes on an mbarrier;
//  - 16 producer warps form P = rho(G) rho*(G') (8 warps, one 4 x 4 (G, G') sub-block each)
//    and w = df / (w + Delta + i eta) (8 warps, 16 columns each) in FP32, with w + Delta
//    carried as (hi, lo) floats so the sum keeps FP64-level accuracy when it cancels, split
//    every value v into v_hi = round16(v) and v_lo = round16(v - v_hi) (FP16 with power-of-two
//    scales, or BF16), and write the tiles MN-major with the 128-byte swizzle (lane = pair =
//    K index; 16-byte chunks of 8 rows or columns), then arrive on the even CTA's barrier;
//  - one thread of the even CTA issues A_hi B_hi + A_hi B_lo + A_lo B_hi for both
//    accumulators and commits to the barriers of both CTAs (multicast);
//  - every `flush` stages four epilogue warps per CTA copy their accumulator rows
//    (tcgen05.ld) to a staging area, hand the tensor memory back, and add the staged values
//    into the FP64 sums C with reductions that return nothing (red.global.add.f64) while the
//    next period runs, so FP32 accumulation never spans more than one period.
// Units of work are (row super-tile pair, column tile, pair range), handed out round-robin to
// the clusters.  Every wait on an mbarrier is bounded; on expiry the kernel sets bit 2 of the
// status word, stops issuing work, waits (bounded) for its own copies and MMAs, and frees its
// tensor memory before returning; cluster barriers at the start and the end keep either CTA
// from touching the other's shared memory before it is set up or after it has left.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "lrt_internal.h"
#include "tc_ptx.cuh"

namespace lrt {
namespace {

constexpr int TM = 128;            // rows per accumulator per CTA (64 row pairs)
constexpr int NACC = 2;            // accumulators (row tiles) per CTA
constexpr int TN = 256;            // MMA N: columns per tile (128 frequencies), shared by the pair
constexpr int TNH = TN / 2;        // B columns built by each CTA of the pair
constexpr int KS = 32;             // pairs (K) per pipeline stage
constexpr int GBLK = 8;            // G per block of the blocked rho layout
constexpr int MAXBLK = 6;          // G blocks one row super-tile may touch
constexpr int RROWS = MAXBLK * GBLK;
constexpr int NPROD = 16;          // producer warps 0..15: 0..7 build A, 8..15 build B
constexpr int WMMA = 16;           // MMA warp
constexpr int WLOAD = 21;          // loader warp
constexpr int NTHREADS = 22 * 32;  // + epilogue warps 17..20 (one per TMEM lane quadrant)
constexpr int CHUNKS_A = 4;        // 16-byte chunks (8 rows) per A warp
constexpr int CHUNKS_B = 2;        // 16-byte chunks (8 columns) per B warp
constexpr int A_BYTES = TM * KS * 2;                 // 8 KB per 16-bit row tile
constexpr int B_BYTES = TNH * KS * 2;                // 8 KB per 16-bit half column tile
constexpr int STAGE_BYTES = NACC * 2 * A_BYTES + 2 * B_BYTES;   // 48 KB
constexpr int A_SBO = (TM / 64) * 1024;              // bytes between 8-pair groups of A
constexpr int B_SBO = (TNH / 64) * 1024;
constexpr int RBLK_BYTES = GBLK * KS * 8;            // one G block of one stage: 2 KB
constexpr int PW_OFF = RROWS * KS * 8;               // pair weights after the rows
constexpr int R_STAGE = PW_OFF + KS * 16;            // rho rows, 32 float4 pair weights
constexpr int NSUB = NACC * 64 / 16;                 // sub-blocks of 16 (G, G') pairs per super-tile
constexpr int kFlushStages = 64;   // FP32 accumulation period: 64 stages = 2048 pairs
constexpr int NCHUNK = NACC * TN / 16;  // 16-column pieces of the accumulators per lane

// One q of a launch: its pair densities, weights, tables and FP64 sums.
struct QDesc {
  const float2* rho;          // blocked [ld/32][gpad][32]
  const float4* pw;           // [np rounded up to 32] {Delta_hi, Delta_lo, df sB, 0}
  const int2* rowtab;         // [n_st * NSUB] ring rows of a sub-block's G quads, or (-1, list)
  const int2* lsttab;         // [n_st * NSUB * 16] ring rows of the (G, G') of list slots
  const int* blk;             // [n_st * MAXBLK] G blocks of the super-tile, -1 padding
  const float4* wtab;         // [n_n * 64] per frequency pair {hi_f, hi_f+1, lo_f, lo_f+1}
                              // (CTA r of a pair builds the columns of pairs 32 r .. 32 r + 31)
  const float2* etab;         // [n_n * 64] eta of both columns of each pair (eta lists only)
  double* C;                  // [n_n * TN][ldr] FP64 sums, column-major
  long long np;
  long long ldr;              // = n_st * NACC * TM
  long long k_per_split;      // multiple of KS
  int gpad;
  int n_ru, n_n, n_split;     // row units, column tiles, pair ranges
  // Row unit r: super-tiles 2 r (CTA 0) and 2 r + 1 (CTA 1), 512 rows; or, when it is a half,
  // super-tile r' shared by the pair, CTA c holding its sub-blocks 4 c .. 4 c + 3 in one
  // accumulator (256 rows): every unit under half_all (r' = r), else only the last one when
  // the super-tile count is odd (r' = 2 r).
  int half_all, half_last;
};

struct Params {
  const QDesc* qd;            // [nq of the launch]
  const int2* units;          // [nunits] (q of the launch, unit within the q), q-major
  int nunits;
  float4* stage;              // [gridDim.x][4 warps][NCHUNK][4][32 lanes] accumulator staging
  int* status;
  int flush;                  // stages per accumulator period
  float eta;
};

using namespace tcx;

struct Unit {
  int st, nt;  // super-tile of CTA 0 (CTA 1 takes st + 1 unless half), column tile
  bool half;   // the pair shares super-tile st: CTA r holds its sub-blocks 4 r .. 4 r + 3
  long long kb, ke;
};
__host__ __device__ __forceinline__ Unit unit_of(const QDesc& D, int u) {
  Unit U;
  int tile = u / D.n_split, ks = u % D.n_split;
  const int ru = tile / D.n_n;
  U.nt = tile % D.n_n;
  U.half = D.half_all || (D.half_last && ru == D.n_ru - 1);
  U.st = D.half_all ? ru : 2 * ru;
  U.kb = (long long)ks * D.k_per_split;
  U.ke = min(D.np, U.kb + D.k_per_split);
  return U;
}

// NS: operand (A/B) stages; NSR: prefetch stages of rho blocks and pair weights.  ME: the
// columns carry their own eta (an eta list: columns (eta, w), eta-major), else P.eta.
template <bool BF, int NS, int NSR, bool ME>
__global__ void __launch_bounds__(NTHREADS, 1) chi0_tc_kernel(Params P) {
  extern __shared__ uint8_t smem_raw[];
  // full[s]: this CTA's producers arrive; in the even CTA also the odd CTA's relay.
  // acc_empty[] is used in the even CTA only (the epilogues of both CTAs arrive on it).
  __shared__ __align__(8) uint64_t full[NS], empty[NS], acc_full, acc_empty[NACC], final_bar;
  __shared__ __align__(8) uint64_t rfull[NSR], rempty[NSR];
  __shared__ uint32_t tmem_base_s;
  __shared__ int2 rowtab_s[NSUB];   // byte offsets of the two G quads of each A warp's sub-block
                                    // (x < 0: the sub-block is a list)
  __shared__ int4 lst_s[NSUB][8];   // a list's 16 (G, G') byte offsets, two pairs per int4
  __shared__ int blk_s[MAXBLK];
  __shared__ int nblk_s;
  __shared__ float4 wtab_s[TNH / 4];
  __shared__ float2 etab_s[TNH / 4];
  __shared__ volatile int abort_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cta_rank();
  const bool leader = rank == 0;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t rbase = base + NS * STAGE_BYTES;          // prefetch ring

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], leader ? NPROD + 1 : NPROD);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < NSR; ++s) {
      mbar_init(&rfull[s], 1);
      mbar_init(&rempty[s], NPROD);
    }
    mbar_init(&acc_full, 1);
    for (int a = 0; a < NACC; ++a) mbar_init(&acc_empty[a], 8);
    mbar_init(&final_bar, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == WMMA) {
    // one warp of each CTA of the pair allocates (tensor memory of both CTAs)
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(NACC * TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();   // both CTAs' barriers initialised before any cross-CTA arrive
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const int nunits = P.nunits;
  const uint32_t idesc = (1u << 4) | ((BF ? 1u : 0u) << 7) | ((BF ? 1u : 0u) << 10) | (1u << 15) |
                         (1u << 16) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)((2 * TM) >> 4) << 24);

  uint32_t it = 0;   // stage counter (producers, loader, MMA)
  uint32_t pc = 0;   // accumulator period counter (MMA and epilogue)
  for (int u = cid; u < nunits; u += ncl) {
    const int2 uu = P.units[u];
    const QDesc& D = P.qd[uu.x];
    const Unit U = unit_of(D, uu.y);
    // this CTA's row super-tile (a half unit: both CTAs on the same one, 4 sub-blocks each,
    // accumulator 0 only)
    const int st = U.half ? U.st : U.st + (int)rank;
    const int sub0 = U.half ? 4 * (int)rank : 0;
    const int nacc = U.half ? 1 : NACC;
    // per-unit tables (row pairs and G blocks of the super-tile, frequencies of the column tile)
    __syncthreads();
    if (threadIdx.x < NSUB) {
      const int w = sub0 + (int)threadIdx.x;   // (w >= NSUB: an unused A warp of a half unit)
      const int2 g = w < NSUB ? D.rowtab[st * NSUB + w] : make_int2(0, 0);
      rowtab_s[threadIdx.x] = make_int2(g.x * KS * 8, g.y * KS * 8);
    }
    if (threadIdx.x < NSUB * 16) {
      const int w = sub0 + (int)threadIdx.x / 16;
      const int2 g = w < NSUB ? D.lsttab[(st * NSUB + w) * 16 + threadIdx.x % 16] : make_int2(0, 0);
      reinterpret_cast<int2*>(&lst_s[0][0])[threadIdx.x] = make_int2(g.x * KS * 8, g.y * KS * 8);
    }
    if (threadIdx.x < TNH / 4) wtab_s[threadIdx.x] = D.wtab[U.nt * 64 + rank * (TNH / 4) + threadIdx.x];
    if (ME && threadIdx.x < TNH / 4)
      etab_s[threadIdx.x] = D.etab[U.nt * 64 + rank * (TNH / 4) + threadIdx.x];
    if (threadIdx.x < MAXBLK) blk_s[threadIdx.x] = D.blk[st * MAXBLK + threadIdx.x];
    if (threadIdx.x == 0) {
      int n = 0;
      while (n < MAXBLK && D.blk[st * MAXBLK + n] >= 0) ++n;
      nblk_s = n;
    }
    __syncthreads();
    if (abort_s) break;
    const int nstage = (int)((U.ke - U.kb + KS - 1) / KS);
    const int nper = (nstage + P.flush - 1) / P.flush;

    if (warp < NPROD) {
      // ---------------- producers ----------------
      // Lane = pair.  A warp w (0..7) owns the sub-block of rows 32 w .. 32 w + 31: for a quad
      // block (G quad a, G quad b) chunk i holds the row pairs (4 a + i, 4 b + j), j = 0..3;
      // for a list chunk i holds its pairs 4 i .. 4 i + 3 (ring rows from lst_s).  B warp w
      // (8..15) owns 8 frequencies (2 chunks of 8 columns) of this CTA's 64.  Padding pairs
      // (beyond the last one) and padding G rows have zero pair densities and weights, so no
      // masking is needed.
      uint32_t sto[CHUNKS_A];   // shared-memory offsets of this lane's 16-byte chunks in a stage
#pragma unroll
      for (int cc = 0; cc < CHUNKS_A; ++cc) {
        if (warp < 8) {
          const int c = CHUNKS_A * warp + cc;
          sto[cc] = (c >> 4) * 2 * A_BYTES + mn_chunk(lane, c & 15, A_SBO);
        } else {
          sto[cc] = NACC * 2 * A_BYTES + mn_chunk(lane, CHUNKS_B * (warp - 8) + (cc & 1), B_SBO);
        }
      }
      const int2 ro = rowtab_s[warp & 7];                      // A warps
      const bool is_list = ro.x < 0;
      const float4* wt = wtab_s + CHUNKS_B * 2 * (warp & 7);   // B warps: 4 frequency pairs
      const float2* et = etab_s + CHUNKS_B * 2 * (warp & 7);
      const float eta2 = P.eta * P.eta;
      uint32_t s = it % NS, ph = (it / NS) & 1, sr = it % NSR, phr = (it / NSR) & 1;
      for (int st_ = 0; st_ < nstage; ++st_) {
        // every lane waits; the vote keeps the warp together if one lane's wait gives up
        if (!__all_sync(0xffffffffu, mbar_wait(&rfull[sr], phr, &abort_s, P.status))) break;
        if (!__all_sync(0xffffffffu, mbar_wait(&empty[s], ph ^ 1, &abort_s, P.status))) break;
        const uint32_t ring = rbase + sr * R_STAGE + stage_token();
        const uint32_t sst = base + s * STAGE_BYTES;
        if (warp < 8 && warp >= 4 * nacc) {
          // a half unit: accumulator 1 is not used, its rows are not built
        } else if (warp < 8 && is_list) {
          // 16 listed (G, G'): two loads per product, the same x conj(y) arithmetic
          const uint32_t rl = ring + lane * 8;
          const int4* lt = lst_s[warp];
#pragma unroll
          for (int cc = 0; cc < CHUNKS_A; ++cc) {
            float v[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int4 o = lt[2 * cc + h];
              const float2 x0 = lds_f2(rl + o.x), y0 = lds_f2(rl + o.y);
              const float2 x1 = lds_f2(rl + o.z), y1 = lds_f2(rl + o.w);
              const float2 p0 = __ffma2_rn(make_float2(y0.x, y0.x), x0,
                                           __fmul2_rn(make_float2(y0.y, y0.y), make_float2(x0.y, -x0.x)));
              const float2 p1 = __ffma2_rn(make_float2(y1.x, y1.x), x1,
                                           __fmul2_rn(make_float2(y1.y, y1.y), make_float2(x1.y, -x1.x)));
              v[4 * h] = p0.x;
              v[4 * h + 1] = p0.y;
              v[4 * h + 2] = p1.x;
              v[4 * h + 3] = p1.y;
            }
            uint4 hi, lo;
            Pack<BF>::split(v, hi, lo);
            st_shared_v4(sst + sto[cc], hi);
            st_shared_v4(sst + sto[cc] + A_BYTES, lo);
          }
        } else if (warp < 8) {
          // rho(4a + i) and rho(4b + j) of this lane's pair; x conj(y) as
          // y.re (x.re, x.im) + y.im (x.im, -x.re) in packed FP32x2
          const uint32_t ra = ring + lane * 8 + ro.x, rb = ring + lane * 8 + ro.y;
          float2 X[4], Xr[4], Yr[4], Yi[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float2 x = lds_f2(ra + i * KS * 8), y = lds_f2(rb + i * KS * 8);
            X[i] = x;
            Xr[i] = make_float2(x.y, -x.x);
            Yr[i] = make_float2(y.x, y.x);
            Yi[i] = make_float2(y.y, y.y);
          }
#pragma unroll
          for (int cc = 0; cc < CHUNKS_A; ++cc) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const float2 pv = __ffma2_rn(Yr[j], X[cc], __fmul2_rn(Yi[j], Xr[cc]));
              v[2 * j] = pv.x;       // Re rho(G) rho*(G')
              v[2 * j + 1] = pv.y;   // Im
            }
            uint4 hi, lo;
            Pack<BF>::split(v, hi, lo);
            st_shared_v4(sst + sto[cc], hi);
            st_shared_v4(sst + sto[cc] + A_BYTES, lo);
          }
        } else {
          // two frequencies per packed FP32x2 operation
          const float4 pw = lds_f4(ring + PW_OFF + lane * 16);
          const float2 dh = make_float2(pw.x, pw.x), dl = make_float2(pw.y, pw.y);
          const float2 df = make_float2(pw.z, pw.z);
          const float2 m = make_float2(-P.eta * pw.z, -P.eta * pw.z);
          const float2 e2 = make_float2(eta2, eta2);
#pragma unroll
          for (int cc = 0; cc < CHUNKS_B; ++cc) {
            float v[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float4 w = wt[2 * cc + h];
              // w + Delta from the hi and lo parts of both
              const float2 x = __fadd2_rn(__fadd2_rn(make_float2(w.x, w.y), dh),
                                          __fadd2_rn(make_float2(w.z, w.w), dl));
              float2 d, mm;
              if constexpr (ME) {
                const float2 e = et[2 * cc + h];                    // eta of both columns
                d = __ffma2_rn(x, x, __fmul2_rn(e, e));
                mm = __fmul2_rn(make_float2(-pw.z, -pw.z), e);
              } else {
                d = __ffma2_rn(x, x, e2);
                mm = m;
              }
              const float2 r = make_float2(rcp_approx(d.x), rcp_approx(d.y));
              const float2 re = __fmul2_rn(__fmul2_rn(df, x), r);   // Re df / (x + i eta)
              const float2 im = __fmul2_rn(mm, r);                  // Im
              v[4 * h] = re.x;
              v[4 * h + 1] = im.x;
              v[4 * h + 2] = re.y;
              v[4 * h + 3] = im.y;
            }
            uint4 hi, lo;
            Pack<BF>::split(v, hi, lo);
            st_shared_v4(sst + sto[cc], hi);
            st_shared_v4(sst + sto[cc] + B_BYTES, lo);
          }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&full[s]);
          mbar_arrive(&rempty[sr]);
        }
        ++it;
        if (++s == NS) { s = 0; ph ^= 1; }
        if (++sr == NSR) { sr = 0; phr ^= 1; }
      }
    } else if (warp == WLOAD) {
      // ---------------- loader: rho blocks and pair weights of each stage ----------------
      if (lane == 0) {
        const int nb = nblk_s;
        const uint32_t bytes = (uint32_t)(nb * RBLK_BYTES + KS * 16);
        const float2* rho = D.rho;
        const float4* pwg = D.pw;
        const long long gpad = D.gpad;
        for (int st_ = 0; st_ < nstage; ++st_, ++it) {
          const int sr = it % NSR;
          if (!mbar_wait(&rempty[sr], ((it / NSR) & 1) ^ 1, &abort_s, P.status)) break;
          const long long p0 = U.kb + (long long)st_ * KS;
          mbar_expect_tx(&rfull[sr], bytes);
          const uint32_t dst = rbase + sr * R_STAGE;
          const float2* src = rho + (size_t)(p0 >> 5) * gpad * KS;
          for (int i = 0; i < nb; ++i)
            bulk_g2s(dst + i * RBLK_BYTES, src + (size_t)blk_s[i] * GBLK * KS, RBLK_BYTES, &rfull[sr]);
          bulk_g2s(dst + PW_OFF, pwg + p0, KS * 16, &rfull[sr]);
        }
      }
      it = __shfl_sync(0xffffffffu, it, 0);
    } else if (warp == WMMA) {
      // ---------------- MMA issuer (even CTA) ----------------
      if (leader) {
        bool ok = true;
        for (int per = 0; per < nper && ok; ++per, ++pc) {
          const int s0 = per * P.flush, s1 = min(nstage, s0 + P.flush);
          for (int st_ = s0; st_ < s1; ++st_, ++it) {
            const int s = it % NS;
            if (lane == 0) ok = mbar_wait(&full[s], (it / NS) & 1, &abort_s, P.status);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            const uint32_t sst = base + s * STAGE_BYTES;
            const uint32_t bH = sst + NACC * 2 * A_BYTES, bL = bH + B_BYTES;
#pragma unroll
            for (int kk = 0; kk < KS / 16; ++kk) {
              const uint64_t dBh = sdesc(bH + kk * 2 * B_SBO, 1024, B_SBO);
              const uint64_t dBl = sdesc(bL + kk * 2 * B_SBO, 1024, B_SBO);
#pragma unroll
              for (int a = 0; a < NACC; ++a) {
                if (st_ == s0 && kk == 0) {
                  // first use of accumulator a in this period: both epilogues must have read it
                  if (lane == 0) ok = mbar_wait(&acc_empty[a], (pc & 1) ^ 1, &abort_s, P.status);
                  ok = __shfl_sync(0xffffffffu, ok, 0);
                  if (!ok) break;
                  tc_fence_after();
                }
                if (lane == 0 && a < nacc) {
                  const uint32_t aH = sst + a * 2 * A_BYTES, aL = aH + A_BYTES;
                  const uint64_t dAh = sdesc(aH + kk * 2 * A_SBO, 1024, A_SBO);
                  const uint64_t dAl = sdesc(aL + kk * 2 * A_SBO, 1024, A_SBO);
                  const uint32_t d = tmem + a * TN;
                  mma2(d, dAh, dBh, idesc, (st_ > s0 || kk > 0) ? 1u : 0u);
                  mma2(d, dAh, dBl, idesc, 1u);
                  mma2(d, dAl, dBh, idesc, 1u);
                }
                __syncwarp();
              }
              if (!ok) break;
            }
            if (!ok) break;
            if (lane == 0) mma_commit_pair(&empty[s]);
            __syncwarp();
          }
          if (!ok) break;
          if (lane == 0) mma_commit_pair(&acc_full);
          __syncwarp();
        }
      } else {
        // odd CTA: relay each stage its producers have completed to the even CTA's full[s]
        // (one cluster-scope arrive per stage instead of one per producer warp)
        const uint32_t full0 = cluster_addr(&full[0], 0);
        for (int st_ = 0; st_ < nstage; ++st_, ++it) {
          const int s = it % NS;
          bool ok = true;
          if (lane == 0) {
            ok = mbar_wait(&full[s], (it / NS) & 1, &abort_s, P.status);
            if (ok) mbar_arrive_cluster(full0 + s * 8);
          }
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (!ok) break;
        }
      }
    } else {
      // ---------------- epilogue ----------------
      // Per period: (1) read this CTA's accumulator rows (tcgen05.ld) into a per-warp staging
      // area in global memory with plain stores and hand each accumulator back (to the even
      // CTA) as soon as it has been read; (2) while the next period runs, add the staged FP32
      // values into the FP64 sums C with reductions that return nothing (red.global.add.f64).
      // Each lane reads back only what it wrote.  C is column-major with ldr >= the super-tile
      // rows and n_n * TN columns, so no bounds checks are needed (padding rows and columns
      // collect values that are never read).
      const int q = warp & 3;            // tensor-memory lane quadrant of this warp
      float4* stg = P.stage + ((size_t)blockIdx.x * 4 + q) * (NCHUNK * 4 * 32) + lane;
      const long long grow0 = (long long)st * (NACC * TM) + sub0 * 32 + q * 32 + lane;
      const size_t ldr = (size_t)D.ldr;
      double* cbase = D.C + (size_t)(U.nt * TN) * ldr;
      const uint32_t acc_empty0 = cluster_addr(&acc_empty[0], 0);
      for (int per = 0; per < nper; ++per, ++pc) {
        bool ok = true;
        if (lane == 0) ok = mbar_wait(&acc_full, pc & 1, &abort_s, P.status);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        tc_fence_after();
#pragma unroll 1
        for (int ch = 0; ch < NCHUNK; ++ch) {
          const int a = ch / (TN / 16), c = ch % (TN / 16);
          if (a >= nacc) {
            // accumulator 1 of a half unit holds nothing: hand it back unread
            if (c == TN / 16 - 1) {
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive_cluster(acc_empty0 + a * 8);
            }
            continue;
          }
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
          float4* d = stg + (size_t)ch * 128;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            d[32 * k] = make_float4(__uint_as_float(r[4 * k]), __uint_as_float(r[4 * k + 1]),
                                    __uint_as_float(r[4 * k + 2]), __uint_as_float(r[4 * k + 3]));
          if (c == TN / 16 - 1) {
            // accumulator a has been read: hand it back
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(acc_empty0 + a * 8);
          }
        }
#pragma unroll 1
        for (int ch = 0; ch < NCHUNK; ++ch) {
          const int a = ch / (TN / 16), c = ch % (TN / 16);
          if (a >= nacc) break;
          const float4* sp = stg + (size_t)ch * 128;
          float4 v[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) v[k] = sp[32 * k];
          double* cp = cbase + (size_t)(c * 16) * ldr + grow0 + a * TM;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            red_add_f64(cp, (double)v[k].x);
            red_add_f64(cp + ldr, (double)v[k].y);
            red_add_f64(cp + 2 * ldr, (double)v[k].z);
            red_add_f64(cp + 3 * ldr, (double)v[k].w);
            cp += 4 * ldr;
          }
        }
      }
    }
    // keep every role on the same unit; an abort stops all of them
    __syncthreads();
  }
  // drain: the loader waits (bounded) for its last bulk copies; the even CTA's MMA warp waits
  // for all its MMAs and for the last commits to have arrived, so that nothing is in flight
  // towards either CTA when the pair meets at the closing cluster barrier
  if (warp == WLOAD && lane == 0) {
    for (uint32_t j = (it > (uint32_t)NSR ? it - NSR : 0u); j < it; ++j)
      mbar_drain(&rfull[j % NSR], (j / NSR) & 1, P.status);
  }
  if (warp == WMMA && leader) {
    if (lane == 0) {
      mma_commit_local(&final_bar);
      mbar_drain(&final_bar, 0, P.status);
      for (uint32_t j = (it > (uint32_t)NS ? it - NS : 0u); j < it; ++j)
        mbar_drain(&empty[j % NS], (j / NS) & 1, P.status);
      if (pc > 0) mbar_drain(&acc_full, (pc - 1) & 1, P.status);
    }
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  if (warp == WMMA)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NACC * TN));
}

// chi0[i][G][G'] from the FP64 sums (C column-major: C[col * ldr + row]).  Tensor column pair
// w (of ncol = n_eta x nw_tc, eta-major) holds internal frequency i = (w / nw_tc) nwi + w % nw_tc
// (the w = 0 column appended after the grid is not a tensor column: nw_tc = nwi - 1 then).
__global__ void chi0_unpack(const double* __restrict__ C, long long ldr,
                            const int* __restrict__ rp_of, int nG, int ncol, int nw_tc, int nwi,
                            double scale, double2* __restrict__ chi0) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long total = (long long)ncol * nG * nG;
  if (t >= total) return;
  int Gp = (int)(t % nG);
  int G = (int)((t / nG) % nG);
  int w = (int)(t / ((long long)nG * nG));
  const long long out = ((long long)(w / nw_tc) * nwi + w % nw_tc) * nG * nG + (long long)G * nG + Gp;
  int rp = rp_of[G * nG + Gp];
  const double* cre = C + (long long)(2 * w) * ldr;       // column Re w
  const double* cim = C + (long long)(2 * w + 1) * ldr;   // column Im w
  double RR = cre[2 * rp], IR = cre[2 * rp + 1], RI = cim[2 * rp], II = cim[2 * rp + 1];
  double2 v;
  if (G <= Gp)
    v = make_double2(RR - II, RI + IR);
  else
    v = make_double2(RR + II, RI - IR);
  chi0[out] = make_double2(scale * v.x, scale * v.y);
}

// {Delta_hi, Delta_lo, df sB, 0} per pair (Delta split so that w + Delta keeps FP64-level
// accuracy when it cancels in FP32); df carries the band weights and the power-of-two scale sB.
__global__ void pair_weights_split(const double* __restrict__ eps, const double* __restrict__ occ,
                                   const double* __restrict__ wgt, int nk, int nb,
                                   float sB, float4* __restrict__ pw) {
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
                        (float)(wgt[kn] * wgt[ikq] * (occ[kn] - occ[ikq]) * sB), 0.f);
  }
}

}  // namespace

// ------------------------------------------------------------------ host side
namespace {

// Kernel variants (ring depths) the tuner chooses from, and the unit sizes (stages per unit).
struct Variant {
  int ns, nsr;
};
constexpr Variant kVariants[] = {{4, 2}, {3, 4}};
constexpr int kNumVariants = 2;
constexpr int kUnitStages[] = {4096, 1024, 16384};
constexpr int kNumUnitStages = 3;

size_t smem_of(int v) {
  return (size_t)kVariants[v].ns * STAGE_BYTES + (size_t)kVariants[v].nsr * R_STAGE + 1024;
}
typedef void (*KernFn)(Params);
KernFn kernel_of(bool bf, int v, bool me) {
  if (me) {
    if (bf) return v == 0 ? chi0_tc_kernel<true, 4, 2, true> : chi0_tc_kernel<true, 3, 4, true>;
    return v == 0 ? chi0_tc_kernel<false, 4, 2, true> : chi0_tc_kernel<false, 3, 4, true>;
  }
  if (bf) return v == 0 ? chi0_tc_kernel<true, 4, 2, false> : chi0_tc_kernel<true, 3, 4, false>;
  return v == 0 ? chi0_tc_kernel<false, 4, 2, false> : chi0_tc_kernel<false, 3, 4, false>;
}

// Per-context state of the tensor path (owned through lrt_ctx::tc).
struct TcState {
  QDesc* d_qdesc = nullptr;
  int qdesc_cap = 0;
  int2* d_units = nullptr;
  int units_cap = 0;
  std::vector<QDesc> qdesc_h;      // what d_qdesc holds
  std::vector<int2> units_h;       // what d_units holds
  float4* stage = nullptr;
  size_t stage_bytes = 0;
  int ncl[2][kNumVariants][2] = {};   // resident CTA pairs per (bf, variant, eta list)
  struct Choice {
    int v, ui, half;   // kernel variant, unit-size index, half row units
  };
  std::map<std::vector<long long>, Choice> tuned;   // shape -> choice
};

TcState* tc_of(const lrt_ctx* c) {
  lrt_ctx* cc = const_cast<lrt_ctx*>(c);
  if (!cc->tc) cc->tc = new TcState();
  return static_cast<TcState*>(cc->tc);
}

lrt_status cluster_capacity(const lrt_ctx* c, bool bf, int v, int* out) {
  TcState* T = tc_of(c);
  const bool me = c->neta > 1;
  if (T->ncl[bf][v][me] > 0) {
    *out = T->ncl[bf][v][me];
    return LRT_OK;
  }
  KernFn kern = kernel_of(bf, v, me);
  const size_t smem = smem_of(v);
  LRT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(NTHREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int dev = 0, nsm = 0, n = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  cfg.gridDim = dim3(2 * (nsm / 2));
  LRT_CUDA(cudaOccupancyMaxActiveClusters(&n, (const void*)kern, &cfg));
  if (n < 1) {
    set_error("the chi0 tensor kernel cannot be resident as a CTA pair");
    return LRT_EUNSUPPORTED;
  }
  T->ncl[bf][v][me] = n;
  *out = n;
  return LRT_OK;
}

}  // namespace

void free_tc_state(lrt_ctx* c) {
  if (!c->tc) return;
  TcState* T = static_cast<TcState*>(c->tc);
  cudaFree(T->d_qdesc);
  cudaFree(T->d_units);
  cudaFree(T->stage);
  delete T;
  c->tc = nullptr;
}

void free_split_plan(SplitPlan& sp) {
  cudaFree(sp.rowtab);
  cudaFree(sp.lsttab);
  cudaFree(sp.blk);
  cudaFree(sp.rp_of);
  cudaFree(sp.wtab);
  cudaFree(sp.etab);
  cudaFree(sp.pw);
  cudaFree(sp.C);
  cudaFree(sp.rho);
  sp = SplitPlan();
}

// Frequencies per eta that run as tensor columns: every internal one except a w = 0 appended
// after the grid (computed by chi0_zero_split_kernel instead).
static int nw_tc(const lrt_ctx* c) { return c->hcol == c->nw ? c->nwi - 1 : c->nwi; }
static int ncol_tc(const lrt_ctx* c) { return c->neta * nw_tc(c); }

// A list costs its A warp about twice a quad block's shared-memory loads and instructions.
// Inside each super-tile the lists take the A warp positions 2, 7, 3, 6, 1, 5, 0, 4 in that
// order: warp w runs on SM sub-partition w % 4, and sub-partition 0 also runs the MMA issuer
// (warp 16), whose issue slots a busy list warp delays; a half unit gives positions 0-3 and
// 4-7 to different CTAs, so its first two lists go one to each.  (Spreading the lists over
// more super-tiles measured slower: a row unit pays for its lists about once, however many.)
// sub is padded to n_st * NSUB entries, (-2, 0) marking a padding slot.
static void seat_lists(int n_st, std::vector<int2>& sub) {
  sub.resize((size_t)n_st * NSUB, make_int2(-2, 0));
  static const int kPos[NSUB] = {2, 7, 3, 6, 1, 5, 0, 4};
  for (int t = 0; t < n_st; ++t) {
    int2* e = &sub[(size_t)t * NSUB];
    std::vector<int2> ls, rest;
    for (int w = 0; w < NSUB; ++w) (e[w].x == -1 ? ls : rest).push_back(e[w]);
    std::vector<char> taken(NSUB, 0);
    for (size_t k = 0; k < ls.size(); ++k) {
      e[kPos[k]] = ls[k];
      taken[kPos[k]] = 1;
    }
    size_t r = 0;
    for (int w = 0; w < NSUB; ++w)
      if (!taken[w]) e[w] = rest[r++];
  }
}

// Row pairs of the Hermitian split in sub-blocks of 16 (G <= G') pairs, in super-tile order
// (NSUB consecutive sub-blocks per super-tile).  A sub-block is either a 4 x 4 block of G
// quads (qa, qb), its pairs (4 qa + i, 4 qb + j), or a list of 16 arbitrary pairs.  A quad
// block costs 8 pair-density loads per lane for its 16 products, a list 32, so quads are used
// wherever they lose nothing: every block of two different full quads is one; the pairs that a
// quad block would cover with padding (the diagonal blocks, whose i > j slots repeat pairs,
// and the blocks of the partial last quad) go into lists, except as many of those blocks as
// fit without raising the super-tile count above ceil(N_G (N_G + 1) / 256), the least any
// covering has.  Sub-blocks are ordered by 8-G block pairs (lists filled in the same order),
// so that a super-tile touches at most MAXBLK G blocks (checked by the caller).
static int plan_subblocks(int nG, std::vector<int2>& sub, std::vector<int2>& lists) {
  sub.clear();
  lists.clear();
  const int nQf = nG / 4, r = nG % 4, nblk = (nG + GBLK - 1) / GBLK;
  const long long npairs = (long long)nG * (nG + 1) / 2;
  const int n_st = (int)((npairs + NSUB * 16 - 1) / (NSUB * 16));
  // quad blocks a list could take instead: diagonal (kind 0), full x partial (1), partial
  // diagonal (2); kept as quads, largest first, while the sub-block count allows
  struct Cand {
    int kind, qa, pairs;
  };
  std::vector<Cand> cands;
  if (r)
    for (int qa = 0; qa < nQf; ++qa) cands.push_back({1, qa, 4 * r});
  for (int qa = 0; qa < nQf; ++qa) cands.push_back({0, qa, 10});
  if (r) cands.push_back({2, nQf, r * (r + 1) / 2});
  std::stable_sort(cands.begin(), cands.end(), [](const Cand& a, const Cand& b) { return a.pairs > b.pairs; });
  const long long nreg = (long long)nQf * (nQf - 1) / 2;
  long long left = npairs - 16 * nreg, nsub = nreg + (left + 15) / 16;
  std::vector<char> keep_diag(nQf + 1, 0), keep_part(nQf + 1, 0);
  for (const Cand& cd : cands) {
    const long long n2 = nsub + 1 - (left + 15) / 16 + (left - cd.pairs + 15) / 16;
    if (n2 > (long long)NSUB * n_st) continue;
    nsub = n2;
    left -= cd.pairs;
    (cd.kind == 1 ? keep_part : keep_diag)[cd.qa] = 1;
  }
  std::vector<int2> pend;
  auto emit = [&](bool all) {
    while (pend.size() >= 16 || (all && !pend.empty())) {
      const int n = std::min<int>(16, (int)pend.size());
      sub.push_back(make_int2(-1, (int)(lists.size() / 16)));
      for (int t = 0; t < 16; ++t) lists.push_back(t < n ? pend[t] : make_int2(-1, -1));
      pend.erase(pend.begin(), pend.begin() + n);
    }
  };
  for (int I = 0; I < nblk; ++I) {
    for (int qa = 2 * I; qa < std::min(nQf, 2 * I + 2); ++qa) {
      if (keep_diag[qa]) {
        sub.push_back(make_int2(qa, qa));
      } else {
        for (int i = 0; i < 4; ++i)
          for (int j = i; j < 4; ++j) pend.push_back(make_int2(4 * qa + i, 4 * qa + j));
      }
    }
    emit(false);
    for (int J = I; J < nblk; ++J)
      for (int qa = 2 * I; qa < 2 * I + 2; ++qa)
        for (int qb = 2 * J; qb < 2 * J + 2; ++qb)
          if (qa < qb && qb < nQf) sub.push_back(make_int2(qa, qb));
    if (r) {
      for (int qa = 2 * I; qa < std::min(nQf, 2 * I + 2); ++qa) {
        if (keep_part[qa]) {
          sub.push_back(make_int2(qa, nQf));
        } else {
          for (int i = 0; i < 4; ++i)
            for (int Gp = 4 * nQf; Gp < nG; ++Gp) pend.push_back(make_int2(4 * qa + i, Gp));
        }
      }
      if (I == (4 * nQf) / GBLK) {
        if (keep_diag[nQf]) {
          sub.push_back(make_int2(nQf, nQf));
        } else {
          for (int G = 4 * nQf; G < nG; ++G)
            for (int Gp = G; Gp < nG; ++Gp) pend.push_back(make_int2(G, Gp));
        }
      }
      emit(false);
    }
  }
  emit(true);
  seat_lists(n_st, sub);
  return n_st;
}

// The row tables of N_G response G vectors: super-tiles, per sub-block its quads' ring rows or
// its list, the list slots' ring rows, the G blocks of each super-tile and the row pair of
// every (G, G').  Host only.
static lrt_status row_tables(int nG, int& n_st, int& n_list, std::vector<int2>& rowtab,
                             std::vector<int2>& lsttab, std::vector<int>& blk, std::vector<int>& rp_of) {
  // Sub-blocks of 16 row pairs (quad blocks and pair lists); sub-block s, slot t holds row
  // pair 16 s + t: a quad block's slot 4 i + j is (4 qa + i, 4 qb + j).  In a diagonal quad
  // block the six slots with i > j repeat pairs held by slots with i < j; like padding G and
  // the padding slots of the last list, their rows are computed and never read.
  std::vector<int2> sub, lists;
  n_st = plan_subblocks(nG, sub, lists);
  const int nsub = (int)sub.size();
  // rowtab: a quad block's ring rows of its two quads, or (-1, list) for a list;
  // lsttab: the ring rows of every list slot's (G, G') (zero for quad blocks)
  rowtab.assign((size_t)n_st * NSUB, make_int2(0, 0));
  lsttab.assign((size_t)n_st * NSUB * 16, make_int2(0, 0));
  blk.assign((size_t)n_st * MAXBLK, -1);
  rp_of.assign((size_t)nG * nG, 0);
  n_list = (int)(lists.size() / 16);
  for (int t = 0; t < n_st; ++t) {
    int* bl = &blk[(size_t)t * MAXBLK];
    int n = 0;
    auto slot = [&](int G) {   // ring row of G (its G block taken into the super-tile)
      const int b = G / GBLK;
      for (int i = 0; i < n; ++i)
        if (bl[i] == b) return i * GBLK + G % GBLK;
      if (n == MAXBLK) return -1;
      bl[n] = b;
      return (n++) * GBLK + G % GBLK;
    };
    for (int w = 0; w < NSUB && t * NSUB + w < nsub; ++w) {
      const int s = t * NSUB + w;
      const int2 qq = sub[s];
      if (qq.x == -2) continue;   // padding slot: quad rows (0, 0), computed and never read
      if (qq.x >= 0) {
        const int la = slot(4 * qq.x), lb = slot(4 * qq.y);
        if (la < 0 || lb < 0) {
          set_error("a row super-tile touches more than 6 G blocks");
          return LRT_EUNSUPPORTED;
        }
        rowtab[s] = make_int2(la, lb);
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) {
            const int G = 4 * qq.x + i, Gp = 4 * qq.y + j;
            if (G >= nG || Gp >= nG || G > Gp) continue;
            rp_of[G * nG + Gp] = rp_of[Gp * nG + G] = s * 16 + 4 * i + j;
          }
      } else {
        rowtab[s] = make_int2(-1, qq.y);
        for (int k = 0; k < 16; ++k) {
          const int2 pr = lists[(size_t)qq.y * 16 + k];
          if (pr.x < 0) continue;   // padding slot: ring row 0 (computed, never read)
          const int la = slot(pr.x), lb = slot(pr.y);
          if (la < 0 || lb < 0) {
            set_error("a row super-tile touches more than 6 G blocks");
            return LRT_EUNSUPPORTED;
          }
          lsttab[(size_t)s * 16 + k] = make_int2(la, lb);
          rp_of[pr.x * nG + pr.y] = rp_of[pr.y * nG + pr.x] = s * 16 + k;
        }
      }
    }
    if (n == 0) bl[0] = 0;
  }
  return LRT_OK;
}

// Tables of one q, built once: row super-tiles (sub-blocks of 16 G pairs), G blocks,
// frequency pairs, the unpack map, and the weight and FP64-sum buffers.
static lrt_status build_plan(const lrt_ctx* c, QData& q) {
  SplitPlan& P = q.sp;
  if (P.built) return LRT_OK;
  const int nG = q.nG;
  if (c->rho_gpad < (nG + GBLK - 1) / GBLK * GBLK) {
    set_error("pair densities are not in the blocked layout");
    return LRT_ESTATE;
  }
  int n_st = 0, n_list = 0;
  std::vector<int2> rowtab, lsttab;
  std::vector<int> blk, rp_of;
  if (lrt_status st = row_tables(nG, n_st, n_list, rowtab, lsttab, blk, rp_of)) return st;
  const int nsub = n_st * NSUB;
  // columns (eta, w), eta-major: column j has the frequency freqs[j % nw_tc] and eta j / nw_tc
  const int nc = ncol_tc(c), nwt = nw_tc(c);
  const int n_n = (2 * nc + TN - 1) / TN;
  std::vector<float4> wtab((size_t)n_n * 64, make_float4(0.f, 0.f, 0.f, 0.f));
  std::vector<float2> etab((size_t)n_n * 64, make_float2(0.f, 0.f));
  for (int j = 0; j < nc; ++j) {
    // frequency pair j / 2 of its column tile: {hi_f, hi_f+1, lo_f, lo_f+1}
    const double f = c->freqs[j % nwt];
    const float h = (float)f, l = (float)(f - (double)h);
    float* w4 = reinterpret_cast<float*>(&wtab[j / 2]);
    w4[j % 2] = h;
    w4[2 + j % 2] = l;
    reinterpret_cast<float*>(&etab[j / 2])[j % 2] = (float)c->etas[j / nwt];
  }
  P.nsub = nsub;
  P.n_st = n_st;
  P.n_n = n_n;
  P.ldc = n_n * TN;
  P.ldr = (long long)n_st * NACC * TM;
  P.pw_n = (size_t)((c->np + KS - 1) / KS * KS);
  auto fail = [&](cudaError_t e) {
    free_split_plan(P);
    set_error(std::string("chi0 plan: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LRT_ENOMEM : LRT_ECUDA;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&P.rowtab, rowtab.size() * sizeof(int2))) != cudaSuccess ||
      (e = cudaMalloc(&P.lsttab, lsttab.size() * sizeof(int2))) != cudaSuccess ||
      (e = cudaMalloc(&P.blk, blk.size() * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&P.rp_of, rp_of.size() * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&P.wtab, wtab.size() * sizeof(float4))) != cudaSuccess ||
      (e = cudaMalloc(&P.etab, etab.size() * sizeof(float2))) != cudaSuccess ||
      (!P.pw && (e = cudaMalloc(&P.pw, P.pw_n * sizeof(float4))) != cudaSuccess) ||
      (e = cudaMalloc(&P.C, (size_t)P.ldr * P.ldc * sizeof(double))) != cudaSuccess)
    return fail(e);
  if ((e = cudaMemcpy(P.rowtab, rowtab.data(), rowtab.size() * sizeof(int2), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(P.lsttab, lsttab.data(), lsttab.size() * sizeof(int2), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(P.blk, blk.data(), blk.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(P.rp_of, rp_of.data(), rp_of.size() * sizeof(int), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(P.wtab, wtab.data(), wtab.size() * sizeof(float4), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(P.etab, etab.data(), etab.size() * sizeof(float2), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemset(P.pw, 0, P.pw_n * sizeof(float4))) != cudaSuccess)
    return fail(e);
  P.built = true;
  return LRT_OK;
}

// power-of-two scales that keep the FP16 low parts clear of the subnormal range: the pair
// densities carry split_rho_scale() (so P carries its square, sA) and df carries sB
static double scale_A(const lrt_ctx* c) {
  const double r = split_rho_scale(c->precision);
  return r * r;
}
// (from the smallest eta of the list: |w| <= df/eta, so every column fits the FP16 range)
static float scale_B(const lrt_ctx* c) {
  if (c->precision == LRT_PREC_BF16X3) return 1.0f;
  return std::ldexp(1.0f, (int)std::floor(std::log2(16384.0 * c->etas[0])));
}

// Units of one q for a target of `stages` per unit (a multiple of the accumulator period).
static void split_q(const lrt_ctx* c, const SplitPlan& P, int stages, int* n_split, long long* kps) {
  const long long nst = (c->np + KS - 1) / KS;
  long long sp = std::max<long long>(1, (nst + stages / 2) / stages);
  long long k = (c->np + sp - 1) / sp;
  k = (k + (long long)KS * kFlushStages - 1) / ((long long)KS * kFlushStages) * ((long long)KS * kFlushStages);
  *kps = k;
  *n_split = (int)((c->np + k - 1) / k);
  (void)P;
}

// Descriptor and unit tables of a launch (q-major), uploaded when they changed.
static lrt_status upload_tables(const lrt_ctx* c, const std::vector<int>& qs,
                                const std::vector<const void*>& rhos, int stages, bool half_all,
                                int limit_units, int* nunits, cudaStream_t s) {
  TcState* T = tc_of(c);
  std::vector<QDesc> qd(qs.size());
  std::vector<int2> units;
  for (size_t i = 0; i < qs.size(); ++i) {
    const QData& q = c->qd[qs[i]];
    const SplitPlan& P = q.sp;
    QDesc& D = qd[i];
    D.rho = (const float2*)rhos[i];
    D.pw = P.pw;
    D.rowtab = P.rowtab;
    D.lsttab = P.lsttab;
    D.blk = P.blk;
    D.wtab = P.wtab;
    D.etab = P.etab;
    D.C = P.C;
    D.np = c->np;
    D.ldr = P.ldr;
    D.gpad = c->rho_gpad;
    D.half_all = half_all ? 1 : 0;
    D.n_ru = half_all ? P.n_st : (P.n_st + 1) / 2;
    D.half_last = (!half_all && P.n_st % 2) ? 1 : 0;
    D.n_n = P.n_n;
    split_q(c, P, stages, &D.n_split, &D.k_per_split);
    // row unit, then pair range, then column tile: the clusters running at the same time
    // share one row unit, so the column tiles of a pair range read the same pair-density
    // blocks (through L2) and only n_n tiles of FP64 sums (1 MB each) are being reduced into
    // at once; ordering by pair range alone keeps all n_ru n_n of them live, which with the
    // staging areas overflows L2
    for (int ru = 0; ru < D.n_ru; ++ru)
      for (int ks = 0; ks < D.n_split; ++ks)
        for (int nt = 0; nt < D.n_n; ++nt)
          units.push_back(make_int2((int)i, (ru * D.n_n + nt) * D.n_split + ks));
  }
  if (limit_units > 0 && (int)units.size() > limit_units) units.resize(limit_units);
  *nunits = (int)units.size();
  const bool same = qd.size() == T->qdesc_h.size() && units.size() == T->units_h.size() &&
                    std::memcmp(qd.data(), T->qdesc_h.data(), qd.size() * sizeof(QDesc)) == 0 &&
                    std::memcmp(units.data(), T->units_h.data(), units.size() * sizeof(int2)) == 0;
  if (same) return LRT_OK;
  if ((int)qd.size() > T->qdesc_cap) {
    cudaFree(T->d_qdesc);
    T->d_qdesc = nullptr;
    T->qdesc_cap = 0;
    LRT_CUDA(cudaMalloc(&T->d_qdesc, qd.size() * sizeof(QDesc)));
    T->qdesc_cap = (int)qd.size();
  }
  if ((int)units.size() > T->units_cap) {
    cudaFree(T->d_units);
    T->d_units = nullptr;
    T->units_cap = 0;
    LRT_CUDA(cudaMalloc(&T->d_units, units.size() * sizeof(int2)));
    T->units_cap = (int)units.size();
  }
  // the host copies stay in the state, so a captured graph may refer to them
  T->qdesc_h = qd;
  T->units_h = units;
  LRT_CUDA(cudaMemcpyAsync(T->d_qdesc, T->qdesc_h.data(), qd.size() * sizeof(QDesc),
                           cudaMemcpyHostToDevice, s));
  LRT_CUDA(cudaMemcpyAsync(T->d_units, T->units_h.data(), units.size() * sizeof(int2),
                           cudaMemcpyHostToDevice, s));
  return LRT_OK;
}

static lrt_status launch_tables(const lrt_ctx* c, bool bf, int v, int nunits, cudaStream_t s,
                                bool timed) {
  TcState* T = tc_of(c);
  int ncl = 0;
  LRT_TRY(cluster_capacity(c, bf, v, &ncl));
  const int grid = 2 * std::min(ncl, std::max(1, nunits));
  const size_t need = (size_t)grid * 4 * NCHUNK * 4 * 32 * sizeof(float4);
  if (T->stage_bytes < need) {
    cudaFree(T->stage);
    T->stage = nullptr;
    T->stage_bytes = 0;
    LRT_CUDA(cudaMalloc(&T->stage, need));
    T->stage_bytes = need;
  }
  Params P;
  P.qd = T->d_qdesc;
  P.units = T->d_units;
  P.nunits = nunits;
  P.stage = T->stage;
  P.status = c->dw.status;
  P.flush = c->fine_accum ? kFlushStages / 2 : kFlushStages;
  P.eta = (float)c->eta;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NTHREADS);
  cfg.dynamicSmemBytes = smem_of(v);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (timed) {
    TimedLaunch tl(c, &c->ev_chi0, s);
    LRT_CUDA(cudaLaunchKernelEx(&cfg, kernel_of(bf, v, c->neta > 1), P));
  } else {
    LRT_CUDA(cudaLaunchKernelEx(&cfg, kernel_of(bf, v, c->neta > 1), P));
  }
  return LRT_OK;
}

// Variant, unit size and row-unit shape for a launch: forced by the caller, tuned once per
// shape (each candidate timed on the first units of the launch), or the defaults.
static lrt_status choose(const lrt_ctx* c, const std::vector<int>& qs,
                         const std::vector<const void*>& rhos, bool bf, cudaStream_t s, int* v,
                         int* ui, bool* half) {
  *v = c->tune_variant >= 0 ? c->tune_variant : 0;
  *ui = 0;
  *half = c->half_tiles;
  if (c->tune_unit_stages > 0) {
    // forced unit size: use it directly (index -1 means "the forced value")
    *ui = -1;
  }
  if (!c->autotune || c->tune_variant >= 0 || c->tune_unit_stages > 0 || c->half_tiles)
    return LRT_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  LRT_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return LRT_OK;   // no timing inside a capture
  TcState* T = tc_of(c);
  std::vector<long long> key = {bf ? 1 : 0, c->np, ncol_tc(c), c->fine_accum ? 1 : 0};
  for (int qi : qs) key.push_back(c->qd[qi].nG);
  auto it = T->tuned.find(key);
  if (it != T->tuned.end()) {
    *v = it->second.v;
    *ui = it->second.ui;
    *half = it->second.half != 0;
    return LRT_OK;
  }
  cudaEvent_t e0, e1;
  LRT_CUDA(cudaEventCreate(&e0));
  LRT_CUDA(cudaEventCreate(&e1));
  double best = 1e300;
  for (int hm = 0; hm < 2; ++hm)
    for (int cv = 0; cv < kNumVariants; ++cv) {
      int ncl = 0;
      LRT_TRY(cluster_capacity(c, bf, cv, &ncl));
      for (int cu = 0; cu < kNumUnitStages; ++cu) {
        int nunits = 0;
        LRT_TRY(upload_tables(c, qs, rhos, kUnitStages[cu], hm == 1, 2 * ncl, &nunits, s));
        // time per super-tile stage (a 32-pair stage of 256 rows per CTA) of the first 2
        // rounds of units, after a warm-up launch
        LRT_TRY(launch_tables(c, bf, cv, nunits, s, false));
        LRT_CUDA(cudaEventRecord(e0, s));
        LRT_TRY(launch_tables(c, bf, cv, nunits, s, false));
        LRT_CUDA(cudaEventRecord(e1, s));
        LRT_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        LRT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        long long work = 0;
        TcState* TT = tc_of(c);
        for (int u = 0; u < nunits; ++u) {
          const QDesc& D = TT->qdesc_h[TT->units_h[u].x];
          const Unit U = unit_of(D, TT->units_h[u].y);
          work += (U.ke - U.kb + KS - 1) / KS * (U.half ? 1 : 2);
        }
        const double per = ms / (double)std::max(1LL, work);
        if (per < best) {
          best = per;
          *v = cv;
          *ui = cu;
          *half = hm == 1;
        }
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  T->tuned[key] = TcState::Choice{*v, *ui, *half ? 1 : 0};
  // the trial launches added into the sums: clear them
  for (int qi : qs) {
    const SplitPlan& P = c->qd[qi].sp;
    LRT_CUDA(cudaMemsetAsync(P.C, 0, (size_t)P.ldr * P.ldc * sizeof(double), s));
  }
  return LRT_OK;
}

// One tensor launch for the q's `qs` (pair densities in rhos[i]), then the unpack of each.
static lrt_status launch_group(const lrt_ctx* c, const std::vector<int>& qs,
                               const std::vector<const void*>& rhos, cudaStream_t s) {
  const bool bf = c->precision == LRT_PREC_BF16X3;
  int v = 0, ui = 0;
  bool half = false;
  LRT_TRY(choose(c, qs, rhos, bf, s, &v, &ui, &half));
  const int stages = ui < 0 ? c->tune_unit_stages : kUnitStages[ui];
  int nunits = 0;
  LRT_TRY(upload_tables(c, qs, rhos, stages, half, 0, &nunits, s));
  LRT_TRY(launch_tables(c, bf, v, nunits, s, true));
  count_launch(c);
  if (c->profiling)
    for (int qi : qs)
      c->timed_cmac += (double)c->qd[qi].nG * c->qd[qi].nG * c->nw * (double)c->np * c->neta;
  const double scale = 2.0 / (c->nk * c->volume) / (scale_A(c) * (double)scale_B(c));
  for (int qi : qs) {
    QData& q = const_cast<lrt_ctx*>(c)->qd[qi];
    const int nG = q.nG;
    long long total = (long long)ncol_tc(c) * nG * nG;
    chi0_unpack<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(q.sp.C, q.sp.ldr, q.sp.rp_of, nG,
                                                               ncol_tc(c), nw_tc(c), c->nwi, scale,
                                                               q.chi0);
    count_launch(c);
    LRT_CUDA(cudaGetLastError());
  }
  const_cast<lrt_ctx*>(c)->last_tc_variant = v;
  const_cast<lrt_ctx*>(c)->last_tc_unit_stages = stages;
  const_cast<lrt_ctx*>(c)->last_tc_rows = half ? 2 * TM : 2 * NACC * TM;
  return LRT_OK;
}

// chi0 at an appended w = 0 for every eta of q (pair densities in rho), on the CUDA cores.

// Split-form pair weights {Delta_hi, Delta_lo, df sB, 0} of q in q.sp.pw (allocated on first
// use) for the engines that need them without the tensor plan; sB is returned.
lrt_status split_pair_weights(const lrt_ctx* c, QData& q, float* sB, cudaStream_t s) {
  *sB = scale_B(c);
  SplitPlan& P = q.sp;
  if (!P.pw) {
    P.pw_n = (size_t)((c->np + KS - 1) / KS * KS);
    LRT_CUDA(cudaMalloc(&P.pw, P.pw_n * sizeof(float4)));
    LRT_CUDA(cudaMemsetAsync(P.pw, 0, P.pw_n * sizeof(float4), s));
  }
  int dev = 0, nsm = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  pair_weights_split<<<4 * nsm, 256, 0, s>>>(q.eps, q.occ, q.wgt, c->nk, c->nb, *sB, P.pw);
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  return LRT_OK;
}

// chi0 of q_begin .. q_end - 1 on the tensor path.  q's whose pair densities fit in their own
// buffers next to the others' run in one launch; the rest run one at a time in the shared
// pair-density buffer.
lrt_status launch_chi0_split_range(lrt_ctx* c, int q_begin, int q_end, cudaStream_t s) {
  if (c->np <= 0) {
    set_error("no pairs to contract");
    return LRT_EINVAL;
  }
  const float sB = scale_B(c);
  const size_t rho_bytes = (size_t)c->rho_gpad * c->rho_ld * sizeof(float2);
  std::vector<int> grp, solo;
  bool fresh = false;
  for (int iq = q_begin; iq < q_end; ++iq) {
    QData& q = c->qd[iq];
    LRT_TRY(build_plan(c, q));
    if (!q.sp.rho && c->multi_q) {
      size_t fr = 0, tot = 0;
      LRT_CUDA(cudaMemGetInfo(&fr, &tot));
      // keep 8 GB free for everything else
      if (fr > rho_bytes + ((size_t)8 << 30)) {
        if (cudaMalloc(&q.sp.rho, rho_bytes) == cudaSuccess) {
          if (cudaMemset(q.sp.rho, 0, rho_bytes) != cudaSuccess) return LRT_ECUDA;
          fresh = true;
        } else {
          cudaGetLastError();
          q.sp.rho = nullptr;
        }
      }
    }
    (q.sp.rho ? grp : solo).push_back(iq);
  }
  if (!solo.empty()) LRT_TRY(ensure_rho(c));
  if (fresh) LRT_CUDA(cudaDeviceSynchronize());   // the zeroed new buffers are ready
  int dev = 0, nsm = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  auto prep = [&](int iq, void* rho) -> lrt_status {
    QData& q = c->qd[iq];
    pair_weights_split<<<4 * nsm, 256, 0, s>>>(q.eps, q.occ, q.wgt, c->nk, c->nb, sB, q.sp.pw);
    count_launch(c);
    LRT_CUDA(cudaGetLastError());
    LRT_TRY(launch_pair_density(c, q, rho, true, s));
    LRT_CUDA(cudaMemsetAsync(q.sp.C, 0, (size_t)q.sp.ldr * q.sp.ldc * sizeof(double), s));
    return LRT_OK;
  };
  if (!grp.empty()) {
    std::vector<const void*> rhos;
    for (int iq : grp) {
      LRT_TRY(prep(iq, c->qd[iq].sp.rho));
      rhos.push_back(c->qd[iq].sp.rho);
    }
    LRT_TRY(launch_group(c, grp, rhos, s));
    for (int iq : grp) {
      LRT_TRY(launch_zero_split(c, c->qd[iq], c->qd[iq].sp.rho, sB, s));
      LRT_TRY(launch_s0(c, c->qd[iq], iq, c->qd[iq].sp.rho, c->qd[iq].sp.pw, sB, s));
    }
  }
  for (int iq : solo) {
    LRT_TRY(prep(iq, c->dw.rho));
    LRT_TRY(launch_group(c, std::vector<int>{iq}, std::vector<const void*>{c->dw.rho}, s));
    // chi0(0) and S(q,0) need this q's pair densities: before the next q overwrites them
    LRT_TRY(launch_zero_split(c, c->qd[iq], c->dw.rho, sB, s));
    LRT_TRY(launch_s0(c, c->qd[iq], iq, c->dw.rho, c->qd[iq].sp.pw, sB, s));
  }
  return LRT_OK;
}

}  // namespace lrt

extern "C" lrt_status lrtddft_row_plan(int nG, int* n_st, int* n_list, int* max_blocks, int32_t* rp) {
  using namespace lrt;
  if (!n_st || !n_list || !max_blocks) {
    set_error("NULL argument");
    return LRT_EINVAL;
  }
  if (nG < 1 || nG > 4096) {
    set_error("nG out of range");
    return LRT_EINVAL;
  }
  int ns = 0, nl = 0;
  std::vector<int2> rowtab, lsttab;
  std::vector<int> blk, rp_of;
  if (lrt_status st = row_tables(nG, ns, nl, rowtab, lsttab, blk, rp_of)) return st;
  int mb = 0;
  for (int t = 0; t < ns; ++t) {
    int n = 0;
    while (n < MAXBLK && blk[(size_t)t * MAXBLK + n] >= 0) ++n;
    mb = std::max(mb, n);
  }
  *n_st = ns;
  *n_list = nl;
  *max_blocks = mb;
  if (rp) std::memcpy(rp, rp_of.data(), rp_of.size() * sizeof(int32_t));
  return LRT_OK;
}
