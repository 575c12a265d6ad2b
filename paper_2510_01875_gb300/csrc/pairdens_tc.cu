// Pair densities on the 5th-generation tensor cores (tcgen05, single CTA per SM) for the
// split-precision path:
//   rho_p(G) = sum_g c*_nk(g) c_n'k+q(idx_G(g)),   p = (k, n, n'),
// with idx_G(g) the position of G1_g + G in the k+q basis (the gather table).  For each
// (k, G) this is a complex GEMM over the plane waves, run as one real GEMM
//   C'[n][n']       = sum_g Re c_nk(g) Re c'_n'(j) + Im c_nk(g) Im c'_n'(j)   = Re rho
//   C'[n][128 + n'] = sum_g Re c_nk(g) Im c'_n'(j) - Im c_nk(g) Re c'_n'(j)   = Im rho
// i.e. A'[n][K] = (Re c_nk | Im c_nk) over K = (g | N_pwp + g) and, for the Re tile, B' rows
// Re c'(j) for K = g and Im c'(j) for K = N_pwp + g; for the Im tile Im c'(j) and -Re c'(j)
// (j = idx_G(g)).  Each (k, G) is two tiles per pair of 128-band blocks (n block, n' block),
// M = 128, N = 128, K = 2 N_pwp; beyond 128 bands the blocks tile the (n, n') square.
//
// Precision.  The tensor core's FP32 accumulation drops bits below the accumulator's last place
// at every update, always toward zero, so an ordinary FP16 hi/lo split loses about one unit in
// the last place per 16 K (a bias, not noise).  Here every coefficient x (|x| <= 1: the orbitals
// have unit norm) is split on a fixed grid instead: hi = rint(2^11 x), an integer of at most 11
// bits (exact in FP16), and the rest r = 2^11 x - hi in [-1/2, 1/2] is carried as a classic FP16
// pair r1 = fp16(2^12 r), r2 = fp16(2^12 r - r1) (about 22 bits of r), plus r11 = fp16(r).
// Every hi hi product is an integer, and by Cauchy-Schwarz every partial sum of them is at most
// |hi_n| |hi_n'| ~ 2^22 in magnitude, so the FP32 accumulator holds each sum exactly.  The small
// products hi (r1 + r2)' + (r1 + r2) hi' + r11 r1' (all at scale 2^34; ~1e-3 of the total) go
// into a second accumulator, whose truncation is ~1e-3 times smaller; the two are added once at
// the end.  A single rounded remainder (lo = fp16(r)) would leave every coefficient with an
// absolute error up to 2^-24, large against small coefficients: the relative error of the small
// interband densities would then be ~10x that of FP32 arithmetic.
//
// Operands: A' depends on k only; a preparation kernel writes it once per q in the exact
// shared-memory tile layout (MN-major, 128-byte swizzle, parts hi, r1, r2, r11), so each 32-K
// stage is one 32 KB bulk copy.  The k+q orbitals are written once per q as split rows (Re | Im)
// of 256 values per part (hi, r1, r2); per stage, gatherer warps load the half of the 32 rows
// idx_G(g) that the tile needs (negated where it needs -Re) and store it into the swizzled B
// tiles.  Two accumulator pairs
// (512 TMEM columns) alternate between tiles, so four epilogue warps write the previous
// tile's Re or Im parts of rho (scaled, into the blocked layout rho[p/32][G][p%32]) while the
// next one runs.  Every wait is bounded; on expiry bit 2 of the status word is set and the kernel
// drains and returns.
#include <algorithm>
#include <cmath>

#include "lrt_internal.h"
#include "tc_ptx.cuh"

namespace lrt {
namespace {

using namespace tcx;

constexpr int PM = 128;                      // bands per tile (M)
constexpr int PN = 128;                      // bands (N) of one tile (its Re or Im part)
constexpr int PROW = 256;                    // values per prepared k+q row: (Re | Im) x bands
constexpr int PK = 32;                       // K per stage
constexpr int PNS = 4;                       // stages in the ring
constexpr int NPA = 4, NPB = 3;              // operand parts: A hi, r1, r2, r11; B hi, r1, r2
constexpr int PA_BYTES = PM * PK * 2;        // 8 KB, one 16-bit A tile
constexpr int PB_BYTES = PN * PK * 2;        // 8 KB
constexpr int PSTAGE = NPA * PA_BYTES + NPB * PB_BYTES;   // 56 KB
constexpr int PA_SBO = (PM / 64) * 1024;
constexpr int PB_SBO = (PN / 64) * 1024;
constexpr int PW_MMA = 0, PW_LOAD = 1, PW_G0 = 2, PW_E0 = 10;   // warps; gatherers 2..9, epilogue 10..13
constexpr int PTHREADS = 14 * 32;
constexpr double kGrid = 2048.0;             // 2^11: hi = rint(kGrid x), r = kGrid x - hi
constexpr double kRest = 4096.0;             // 2^12: r1 = fp16(kRest r), r2 = fp16(kRest r - r1)
constexpr float kSmall = 1.0f / 4096.0f;     // small-product accumulator (scale 2^34) -> 2^22

// Fixed-grid split of 8 coefficients (already multiplied by kGrid): part[0] hi, part[1] r1,
// part[2] r2, part[3] r11, each 8 x FP16.
__device__ __forceinline__ void grid_split(const double* x, uint4* part) {
  uint32_t o[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double hv[2], rv[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      hv[e] = rint(x[2 * i + e]);
      rv[e] = x[2 * i + e] - hv[e];   // exact
    }
    __half2 h = __floats2half2_rn((float)hv[0], (float)hv[1]);   // integers <= 2^11: exact
    const double s0 = rv[0] * kRest, s1 = rv[1] * kRest;
    __half2 r1 = __floats2half2_rn((float)s0, (float)s1);
    const float2 r1f = __half22float2(r1);
    __half2 r2 = __floats2half2_rn((float)(s0 - (double)r1f.x), (float)(s1 - (double)r1f.y));
    __half2 r11 = __floats2half2_rn((float)rv[0], (float)rv[1]);
    o[0][i] = *reinterpret_cast<uint32_t*>(&h);
    o[1][i] = *reinterpret_cast<uint32_t*>(&r1);
    o[2][i] = *reinterpret_cast<uint32_t*>(&r2);
    o[3][i] = *reinterpret_cast<uint32_t*>(&r11);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) part[j] = make_uint4(o[j][0], o[j][1], o[j][2], o[j][3]);
}

struct PParams {
  const uint4* A;             // [nk][nbt][nst][hi | r1 | r2 | r11 tile] prepared A' (32 KB per stage)
  const uint4* B;             // [nk][nbt][npw + 1][hi | r1 | r2][PROW fp16] k+q rows, last row zero
  const int32_t* gather;      // [nk][nG][npw]
  float2* rho;                // blocked [ld/32][gpad][32]
  int* status;
  int nk, nb, nbt, nG, npw, npwp, nst, gpad;   // nbt: 128-band blocks
  float scale;                // applied to C' when storing rho
};

// Tile t of the launch: part t % 2 (0: Re rho, 1: Im rho) of band blocks (tn, tm) of (k, G),
// with t / 2 = ((k nG + G) nbt + tn) nbt + tm.
struct PTile {
  int k, G, tn, tm, part;
};
__device__ __forceinline__ PTile ptile(const PParams& P, int t) {
  PTile r;
  r.part = t & 1;
  int u = t >> 1;
  r.tm = u % P.nbt;
  u /= P.nbt;
  r.tn = u % P.nbt;
  u /= P.nbt;
  r.G = u % P.nG;
  r.k = u / P.nG;
  return r;
}

// A'[k][band block][stage][part]: thread per (k, block, stage, K in stage, chunk of 8 bands).
__global__ void pd_prep_a(const double2* __restrict__ ck, int nk, int nb, int nbt, int npw, int npwp,
                          int nst, uint4* __restrict__ A) {
  const long long total = (long long)nk * nbt * nst * PK * (PM / 8);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t % (PM / 8));
    const int kk = (int)((t / (PM / 8)) % PK);
    const int s = (int)((t / (PM / 8 * PK)) % nst);
    const long long kb = t / ((long long)PM / 8 * PK * nst);   // k nbt + block
    const int k = (int)(kb / nbt), tb = (int)(kb % nbt);
    const int K = s * PK + kk;
    const bool im = K >= npwp;
    const int g = im ? K - npwp : K;
    double v[8];
    for (int i = 0; i < 8; ++i) {
      const int n = tb * PM + 8 * c + i;
      double x = 0.0;
      if (n < nb && g < npw) {
        const double2 z = ck[((size_t)k * nb + n) * npw + g];
        x = (im ? z.y : z.x) * kGrid;
      }
      v[i] = x;
    }
    uint4 part[4];
    grid_split(v, part);
    uint8_t* tile = reinterpret_cast<uint8_t*>(A) + ((size_t)kb * nst + s) * NPA * PA_BYTES;
#pragma unroll
    for (int j = 0; j < NPA; ++j)
      *reinterpret_cast<uint4*>(tile + j * PA_BYTES + mn_chunk(kk, c, PA_SBO)) = part[j];
  }
}

// k+q rows: thread per (k, band block, row j, chunk of 8 columns); row npw is zero.
__global__ void pd_prep_b(const double2* __restrict__ ckq, int nk, int nb, int nbt, int npw,
                          uint4* __restrict__ B) {
  const long long total = (long long)nk * nbt * (npw + 1) * (PROW / 8);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t % (PROW / 8));
    const int j = (int)((t / (PROW / 8)) % (npw + 1));
    const long long kb = t / ((long long)(PROW / 8) * (npw + 1));   // k nbt + block
    const int k = (int)(kb / nbt), tb = (int)(kb % nbt);
    double v[8];
    for (int i = 0; i < 8; ++i) {
      const int col = 8 * c + i;
      const int n = tb * PM + (col & (PM - 1));
      double x = 0.0;
      if (n < nb && j < npw) {
        const double2 z = ckq[((size_t)k * nb + n) * npw + j];
        x = (col < PM ? z.x : z.y) * kGrid;
      }
      v[i] = x;
    }
    uint4 part[4];
    grid_split(v, part);
    uint4* row = B + ((size_t)kb * (npw + 1) + j) * (NPB * PROW / 8);
#pragma unroll
    for (int p = 0; p < NPB; ++p) row[p * (PROW / 8) + c] = part[p];
  }
}

__device__ __forceinline__ uint4 neg16(uint4 v) {   // negate 8 packed fp16 values
  return make_uint4(v.x ^ 0x80008000u, v.y ^ 0x80008000u, v.z ^ 0x80008000u, v.w ^ 0x80008000u);
}

__global__ void __launch_bounds__(PTHREADS, 1) pair_density_tc_kernel(PParams P) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[PNS], empty[PNS], acc_full[2], acc_empty[2], final_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < PNS; ++s) {
      mbar_init(&full[s], 1 + 4);   // the loader's expect_tx arrive + 4 gatherer warps
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(&final_bar, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == PW_MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(4 * PN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  const int ntiles = 2 * P.nk * P.nG * P.nbt * P.nbt;   // (k, G, n block, n' block, Re | Im)
  const int nst = P.nst;
  const uint32_t idesc = (1u << 4) | (1u << 15) | (1u << 16) | ((uint32_t)(PN >> 3) << 17) |
                         ((uint32_t)(PM >> 4) << 24);
  // tile t: (k, G) = t / 2 as k nG + G, part t % 2 (0: Re rho, 1: Im rho)

  if (warp == PW_LOAD) {
    // ---------------- A' stages: one 16 KB bulk copy each ----------------
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const PTile T = ptile(P, t);
        const size_t kb = (size_t)T.k * P.nbt + T.tn;
        for (int s = 0; s < nst; ++s, ++it) {
          const int slot = it % PNS;
          if (!(ok = mbar_wait(&empty[slot], ((it / PNS) & 1) ^ 1, &abort_s, P.status))) break;
          mbar_expect_tx(&full[slot], NPA * PA_BYTES);
          bulk_g2s(base + slot * PSTAGE,
                   reinterpret_cast<const uint8_t*>(P.A) + (kb * nst + s) * NPA * PA_BYTES,
                   NPA * PA_BYTES, &full[slot]);
        }
      }
      // wait (bounded) for the last copies before the shared memory goes away
      for (uint32_t j = (it > (uint32_t)PNS ? it - PNS : 0u); j < it; ++j)
        mbar_drain(&full[j % PNS], (j / PNS) & 1, P.status);
    }
  } else if (warp >= PW_G0 && warp < PW_E0) {
    // ---------------- gatherers: group (warp - 2) / 4 takes every other stage ----------------
    const int grp = (warp - PW_G0) >> 2, gt = (threadIdx.x - PW_G0 * 32) & 127;
    const int kk = gt >> 2, c0 = (gt & 3) * 4;   // this thread's K row in the stage and 4 chunks
    uint32_t it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const PTile T = ptile(P, t);
      const int part = T.part;
      const int32_t* tab = P.gather + ((size_t)T.k * P.nG + T.G) * P.npw;
      const uint4* Bk = P.B + ((size_t)T.k * P.nbt + T.tm) * (P.npw + 1) * (NPB * PROW / 8);
      for (int s = 0; s < nst; ++s, ++it) {
        if ((int)(it & 1) != grp) continue;
        const int slot = it % PNS;
        if (!__all_sync(0xffffffffu, mbar_wait(&empty[slot], ((it / PNS) & 1) ^ 1, &abort_s, P.status))) {
          ok = false;
          break;
        }
        const int K = s * PK + kk;
        const bool im = K >= P.npwp;
        const int g = im ? K - P.npwp : K;
        int j = g < P.npw ? tab[g] : -1;
        if (j < 0) j = P.npw;                    // the zero row
        const uint4* row = Bk + (size_t)j * (NPB * PROW / 8);
        // Re tile: Re c' (first K half), Im c' (second); Im tile: Im c', then -Re c'
        const int off = (part ^ (im ? 1 : 0)) ? PN / 8 : 0;
        const bool neg = part && im;
        uint4 v[NPB][4];
#pragma unroll
        for (int p = 0; p < NPB; ++p)
#pragma unroll
          for (int i = 0; i < 4; ++i) v[p][i] = row[p * (PROW / 8) + off + c0 + i];
        const uint32_t bt = base + slot * PSTAGE + NPA * PA_BYTES;
#pragma unroll
        for (int p = 0; p < NPB; ++p)
#pragma unroll
          for (int i = 0; i < 4; ++i)
            st_shared_v4(bt + p * PB_BYTES + mn_chunk(kk, c0 + i, PB_SBO), neg ? neg16(v[p][i]) : v[p][i]);
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[slot]);
      }
    }
  } else if (warp == PW_MMA) {
    // ---------------- MMA issuer ----------------
    uint32_t it = 0, tc = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tc) {
      const int buf = tc & 1;
      if (lane == 0) ok = mbar_wait(&acc_empty[buf], ((tc >> 1) & 1) ^ 1, &abort_s, P.status);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc_fence_after();
      const uint32_t d = tmem + buf * 2 * PN, dsm = d + PN;   // hi hi | small products
      for (int s = 0; s < nst; ++s, ++it) {
        const int slot = it % PNS;
        if (lane == 0) ok = mbar_wait(&full[slot], (it / PNS) & 1, &abort_s, P.status);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        tc_fence_after();
        if (lane == 0) {
          const uint32_t sa = base + slot * PSTAGE, sb = sa + NPA * PA_BYTES;
#pragma unroll
          for (int kq = 0; kq < PK / 16; ++kq) {
            uint64_t dA[NPA], dB[NPB];
#pragma unroll
            for (int p = 0; p < NPA; ++p) dA[p] = sdesc(sa + p * PA_BYTES + kq * 2 * PA_SBO, 1024, PA_SBO);
#pragma unroll
            for (int p = 0; p < NPB; ++p) dB[p] = sdesc(sb + p * PB_BYTES + kq * 2 * PB_SBO, 1024, PB_SBO);
            const uint32_t acc = (s > 0 || kq > 0) ? 1u : 0u;
            mma1(d, dA[0], dB[0], idesc, acc);     // hi hi (exact)
            mma1(dsm, dA[0], dB[1], idesc, acc);   // hi r1'
            mma1(dsm, dA[0], dB[2], idesc, 1u);    // hi r2'
            mma1(dsm, dA[1], dB[0], idesc, 1u);    // r1 hi'
            mma1(dsm, dA[2], dB[0], idesc, 1u);    // r2 hi'
            mma1(dsm, dA[3], dB[1], idesc, 1u);    // r11 r1'
          }
          mma1_commit(&empty[slot]);
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
    // ---------------- epilogue: tensor memory -> rho (blocked layout) ----------------
    const int q = warp & 3;
    const int n = q * 32 + lane;   // band n of the nk state (row of the tile)
    uint32_t tc = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tc) {
      const int buf = tc & 1;
      bool ok = true;
      if (lane == 0) ok = mbar_wait(&acc_full[buf], (tc >> 1) & 1, &abort_s, P.status);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc_fence_after();
      const PTile T = ptile(P, t);
      const int G = T.G, nn = T.tn * PM + n;
      const long long p0 = ((long long)T.k * P.nb + nn) * P.nb + (long long)T.tm * PN;
      float* out = reinterpret_cast<float*>(P.rho) + T.part;
#pragma unroll 1
      for (int c = 0; c < PN / 16; ++c) {
        uint32_t big[16], sml[16];   // the two accumulators' columns 16 c .. 16 c + 15
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + buf * 2 * PN + c * 16;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15}, [%16];"
            : "=r"(big[0]), "=r"(big[1]), "=r"(big[2]), "=r"(big[3]), "=r"(big[4]), "=r"(big[5]),
              "=r"(big[6]), "=r"(big[7]), "=r"(big[8]), "=r"(big[9]), "=r"(big[10]), "=r"(big[11]),
              "=r"(big[12]), "=r"(big[13]), "=r"(big[14]), "=r"(big[15])
            : "r"(ta));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15}, [%16];"
            : "=r"(sml[0]), "=r"(sml[1]), "=r"(sml[2]), "=r"(sml[3]), "=r"(sml[4]), "=r"(sml[5]),
              "=r"(sml[6]), "=r"(sml[7]), "=r"(sml[8]), "=r"(sml[9]), "=r"(sml[10]), "=r"(sml[11]),
              "=r"(sml[12]), "=r"(sml[13]), "=r"(sml[14]), "=r"(sml[15])
            : "r"(ta + PN));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (nn < P.nb) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int np_ = c * 16 + j;
            if (T.tm * PN + np_ < P.nb) {
              const long long p = p0 + np_;
              out[2 * (((size_t)((p >> 5) * P.gpad + G) << 5) + (size_t)(p & 31))] =
                  __fmaf_rn(__uint_as_float(sml[j]), kSmall, __uint_as_float(big[j])) * P.scale;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == PW_MMA)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * PN));
}

}  // namespace

// Tensor-core pair densities of one q into the blocked FP32 layout (any band count: the
// (n, n') square is tiled by 128-band blocks).
lrt_status launch_pair_density_tc(const lrt_ctx* c, const QData& q, void* rho, cudaStream_t s) {
  const int nbt = (c->nb + PM - 1) / PM;
  const int npw = c->npw;
  const int npwp = (npw + PK - 1) / PK * PK;
  const int nst = 2 * npwp / PK;
  lrt_ctx* cc = const_cast<lrt_ctx*>(c);
  const size_t a_bytes = (size_t)c->nk * nbt * nst * NPA * PA_BYTES;
  const size_t b_bytes = (size_t)c->nk * nbt * (npw + 1) * NPB * PROW * 2;
  if (cc->dw.pd_bytes < a_bytes + b_bytes) {
    cudaFree(cc->dw.pd_work);
    cc->dw.pd_work = nullptr;
    cc->dw.pd_bytes = 0;
    LRT_CUDA(cudaMalloc(&cc->dw.pd_work, a_bytes + b_bytes));
    cc->dw.pd_bytes = a_bytes + b_bytes;
  }
  uint4* A = reinterpret_cast<uint4*>(cc->dw.pd_work);
  uint4* B = reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(cc->dw.pd_work) + a_bytes);
  int dev = 0, nsm = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const double2* ck = q.coeff;
  const double2* ckq = q.coeff + (size_t)c->nk * c->nb * npw;
  pd_prep_a<<<8 * nsm, 256, 0, s>>>(ck, c->nk, c->nb, nbt, npw, npwp, nst, A);
  pd_prep_b<<<8 * nsm, 256, 0, s>>>(ckq, c->nk, c->nb, nbt, npw, B);
  count_launch(c, 2);
  LRT_CUDA(cudaGetLastError());
  PParams P;
  P.A = A;
  P.B = B;
  P.gather = q.gather;
  P.rho = (float2*)rho;
  P.status = c->dw.status;
  P.nk = c->nk;
  P.nb = c->nb;
  P.nbt = nbt;
  P.nG = q.nG;
  P.npw = npw;
  P.npwp = npwp;
  P.nst = nst;
  P.gpad = c->rho_gpad;
  P.scale = (float)(split_rho_scale(c->precision) / (kGrid * kGrid));
  const size_t smem = (size_t)PNS * PSTAGE + 1024;
  // raised once per device (repeated calls and graph captures make no attribute call)
  static size_t attr_set[64] = {0};
  if (dev < 0 || dev >= 64 || attr_set[dev] < smem) {
    LRT_CUDA(cudaFuncSetAttribute(pair_density_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    if (dev >= 0 && dev < 64) attr_set[dev] = smem;
  }
  const int grid = (int)std::min<long long>(nsm, 2LL * c->nk * q.nG * nbt * nbt);
  {
    TimedLaunch tl(c, &c->ev_rho, s);
    pair_density_tc_kernel<<<grid, PTHREADS, smem, s>>>(P);
  }
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  return LRT_OK;
}

}  // namespace lrt
