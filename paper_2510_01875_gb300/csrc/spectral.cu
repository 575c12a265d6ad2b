// chi0 through a spectral function on a grid of transition energies (an engine variant the
// paper does not use; it takes the number of frequencies out of the cost of the pair sum).
//
// With x_p = -Delta_p = eps_n'k+q - eps_nk, each pole 1/(w - x_p + i eta) of the Adler-Wiser sum
// is replaced by its order-m Lagrange interpolant in x_p on the grid x_b = x_0 + b h:
//     A_b(G,G')   = sum_p P_p(G,G') df_p L_b(x_p),      P_p = rho_p(G) rho_p*(G')
//     chi0_GG'(w) = (2/(N_k Omega)) sum_b A_b(G,G') / (w - x_b + i eta),
// so the error is that of order-m interpolation, O((h/eta)^(m+1)) relative (m = 1 or 3).
// The pair sum runs once for all frequencies and broadenings:
//  1. per pair its bin j (x_j <= x_p < x_j+1) and fraction f; pairs with df = 0 drop out;
//  2. a counting sort of the pairs by bin;
//  3. per bin the moments M_k(j) = sum_{p in bin j} P_p df_p f_p^k (k = 0..m) of every G <= G'
//     pair, one block per run of whole bins, the pair densities gathered in sorted order into
//     shared memory; FP64 for the FP64 form, FP32 products with compensated FP32 sums for the
//     split forms (whose pair densities are FP32);
//  4. A_b from the moments (L_c(f) is a polynomial in f: A_b = sum_c sum_k a_ck M_k(j(b, c)));
//  5. the transform as a real GEMM (cuBLAS): rows Re A, Im A of every G <= G' pair, columns
//     Re, Im of 1/(w - x_b + i eta) of every (eta, w) column, inner dimension the bins; FP64
//     (DGEMM) for the FP64 form, FP32 products summed over 256 bins at a time and the chunks in
//     FP64 for the split forms;
//  6. unpack with the Hermitian split of P (chi0(G',G) from conj A).
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "lrt_internal.h"
#include "tc_ptx.cuh"

namespace lrt {
namespace {

using namespace tcx;

// Block shape of the moments kernel: the FP32 form (split contexts) keeps its compensated bin
// totals in shared memory and runs 32 warps of 2 G <= G' pairs each; the FP64 form keeps them
// in registers, 8 warps of 4 pairs each.  Either way a block covers 2048 or 1024 of the pairs.
template <typename T>
struct SpCfg;
template <>
struct SpCfg<float> {
  static constexpr int threads = 1024, E = 2;
};
template <>
struct SpCfg<double> {
  static constexpr int threads = 256, E = 4;
};
constexpr int SP_KCHUNK = 256;                   // bins per FP32 partial product of the transform

// Lagrange basis of order m as polynomials in the fraction f: L_c(f) = sum_k a[c][k] f^k.
// m = 1: nodes j, j + 1.  m = 3: nodes j - 1 .. j + 2.
__constant__ double kLag1[2][2] = {{1.0, -1.0}, {0.0, 1.0}};
__constant__ double kLag3[4][4] = {{0.0, -1.0 / 3.0, 0.5, -1.0 / 6.0},
                                   {1.0, -0.5, -1.0, 0.5},
                                   {0.0, 1.0, 0.5, -0.5},
                                   {0.0, -1.0 / 6.0, 0.0, 1.0 / 6.0}};

// x_p and df_p of every pair (k, n, n') in the order of the pair densities.
__global__ void sp_pairs(const double* __restrict__ eps, const double* __restrict__ occ,
                         const double* __restrict__ wgt, int nk, int nb, double* __restrict__ x,
                         double* __restrict__ df) {
  const long long np = (long long)nk * nb * nb;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(p % nb);
    const long long kn = p / nb;
    const int k = (int)(kn / nb);
    const size_t ikq = (size_t)(nk + k) * nb + m;
    x[p] = eps[ikq] - eps[kn];
    df[p] = wgt[kn] * wgt[ikq] * (occ[kn] - occ[ikq]);
  }
}

__device__ __forceinline__ unsigned long long ord_key(double v) {
  // order-preserving map of a double onto unsigned integers (for atomicMin / atomicMax)
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__host__ __device__ inline double ord_val(unsigned long long k) {
  const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  std::memcpy(&d, &u, sizeof d);
  return d;
#endif
}

// min and max of x over the pairs with df != 0 (mm[0] = key of min, mm[1] = key of max)
__global__ void sp_range(const double* __restrict__ x, const double* __restrict__ df, long long np,
                         unsigned long long* __restrict__ mm) {
  unsigned long long lo = ~0ull, hi = 0ull;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x)
    if (df[p] != 0.0) {
      const unsigned long long k = ord_key(x[p]);
      lo = min(lo, k);
      hi = max(hi, k);
    }
  for (int o = 16; o; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&mm[0], lo);
    atomicMax(&mm[1], hi);
  }
}

// bin of every pair (-1: df = 0) and the bin histogram
__global__ void sp_bins(const double* __restrict__ x, const double* __restrict__ df, long long np,
                        double x0, double h, int* __restrict__ bin, int* __restrict__ count) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    int j = -1;
    if (df[p] != 0.0) {
      j = (int)floor((x[p] - x0) / h);
      atomicAdd(&count[j], 1);
    }
    bin[p] = j;
  }
}

// pairs in bin order: perm[pos] = p, and per sorted position the moment coefficients
// df f^k (k = 0..m) and the bin
template <typename T, int M>
__global__ void sp_scatter(const double* __restrict__ x, const double* __restrict__ df,
                           const int* __restrict__ bin, long long np, double x0, double h,
                           int* __restrict__ cursor, int* __restrict__ perm, int* __restrict__ sbin,
                           T* __restrict__ coef) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    const int j = bin[p];
    if (j < 0) continue;
    const int pos = atomicAdd(&cursor[j], 1);
    perm[pos] = (int)p;
    sbin[pos] = j;
    const double f = (x[p] - x0) / h - (double)j;
    double fk = df[p];
#pragma unroll
    for (int k = 0; k <= M; ++k) {
      coef[(size_t)pos * (M + 1) + k] = (T)fk;
      fk *= f;
    }
  }
}

template <typename T>
struct V2;
template <>
struct V2<float> {
  using type = float2;
};
template <>
struct V2<double> {
  using type = double2;
};

// compensated (Kahan) accumulation for the FP32 sums; plain for FP64
template <typename T>
__device__ __forceinline__ void kadd(T& s, T& c, T v) {
  if constexpr (sizeof(T) == 4) {
    const T y = v - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  } else {
    s += v;
  }
}

// Moments of whole bins: block b takes the sorted positions [range[b].x, range[b].y) (whole
// bins) and threads x E of the G <= G' pairs (blockIdx.y).  rho: FP64 [G][ld] (T = double) or the
// split form's blocked FP32 [p/32][gpad][32] (T = float, values scaled by a power of two that
// the caller removes).  Mom [nbins][M + 1][ngg] complex FP64.
template <typename T, int M, int CH>   // CH: sorted pairs per staged chunk
__global__ void __launch_bounds__(SpCfg<T>::threads, 1) sp_moments(
    const void* __restrict__ rho_v, long long ld, int gpad, int nG, int ngg,
    const int* __restrict__ perm, const int* __restrict__ sbin, const T* __restrict__ coef,
    const int2* __restrict__ range, double2* __restrict__ Mom) {
  using T2 = typename V2<T>::type;
  constexpr int NT = SpCfg<T>::threads, SP_E = SpCfg<T>::E, SP_TILE = NT * SP_E;
  constexpr bool F32 = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char sp_smem[];
  // two buffers of [CH pairs][nG] pair densities (pair-major, so the lanes of a warp, which
  // hold consecutive G <= G' pairs, read consecutive G' without bank conflicts), [CH][M + 1]
  // moment coefficients and [CH] bins: chunk c + 1 arrives by asynchronous copies while chunk
  // c is summed
  const size_t bufsz = (size_t)CH * nG * sizeof(T2) + CH * (M + 1) * sizeof(T) + CH * sizeof(int);
  // FP32 form: the compensated bin totals (sum re, sum im, compensation re, im) of every
  // (pair, k) of this thread, [SP_E (M + 1) 4][NT], after the two chunk buffers
  float* tot = reinterpret_cast<float*>(sp_smem + 2 * bufsz);
  const int tid = threadIdx.x;
  const int2 rg = range[blockIdx.x];
  // this thread's G <= G' pairs (row-major upper triangle)
  int ga[SP_E], gb[SP_E];
#pragma unroll
  for (int e = 0; e < SP_E; ++e) {
    const int idx = blockIdx.y * SP_TILE + e * NT + tid;
    ga[e] = -1;
    gb[e] = 0;
    if (idx < ngg) {
      int G = 0, rem = idx;
      while (rem >= nG - G) {
        rem -= nG - G;
        ++G;
      }
      ga[e] = G;
      gb[e] = G + rem;
    }
  }
  T2 pp[SP_E][M + 1];                   // this chunk's partial sums (re, im)
  T sr[SP_E][M + 1], si[SP_E][M + 1];   // FP64 form: the bin totals
  auto tref = [&](int e, int k, int j) -> float& { return tot[((e * (M + 1) + k) * 4 + j) * NT + tid]; };
  auto zero_totals = [&]() {
#pragma unroll
    for (int e = 0; e < SP_E; ++e)
#pragma unroll
      for (int k = 0; k <= M; ++k) {
        if constexpr (F32) {
#pragma unroll
          for (int j = 0; j < 4; ++j) tref(e, k, j) = 0.f;
        } else {
          sr[e][k] = si[e][k] = 0;
        }
      }
  };
#pragma unroll
  for (int e = 0; e < SP_E; ++e)
#pragma unroll
    for (int k = 0; k <= M; ++k) pp[e][k].x = pp[e][k].y = 0;
  zero_totals();
  int cur = -1;
  auto fold = [&]() {
#pragma unroll
    for (int e = 0; e < SP_E; ++e)
#pragma unroll
      for (int k = 0; k <= M; ++k) {
        if constexpr (F32) {
          float s0 = tref(e, k, 0), s1 = tref(e, k, 1), c0 = tref(e, k, 2), c1 = tref(e, k, 3);
          kadd(s0, c0, (float)pp[e][k].x);
          kadd(s1, c1, (float)pp[e][k].y);
          tref(e, k, 0) = s0;
          tref(e, k, 1) = s1;
          tref(e, k, 2) = c0;
          tref(e, k, 3) = c1;
        } else {
          sr[e][k] += pp[e][k].x;
          si[e][k] += pp[e][k].y;
        }
        pp[e][k].x = pp[e][k].y = 0;
      }
  };
  auto flush = [&]() {
    fold();
    if (cur >= 0) {
#pragma unroll
      for (int e = 0; e < SP_E; ++e) {
        if (ga[e] < 0) continue;
        const int idx = blockIdx.y * SP_TILE + e * NT + tid;
#pragma unroll
        for (int k = 0; k <= M; ++k) {
          double2 v;
          if constexpr (F32)
            v = make_double2((double)tref(e, k, 0) - (double)tref(e, k, 2),
                             (double)tref(e, k, 1) - (double)tref(e, k, 3));
          else
            v = make_double2((double)sr[e][k], (double)si[e][k]);
          Mom[((size_t)cur * (M + 1) + k) * ngg + idx] = v;
        }
      }
    }
    zero_totals();
  };
  const int nchunk = (rg.y - rg.x + CH - 1) / CH;
  auto issue = [&](int ck) {
    const int i0 = rg.x + ck * CH, n = min(CH, rg.y - i0);
    unsigned char* bufp = sp_smem + (size_t)(ck & 1) * bufsz;
    const uint32_t rdst = smem_u32(bufp);
    const uint32_t cdst = rdst + (uint32_t)(CH * nG * sizeof(T2));
    const uint32_t bdst = cdst + (uint32_t)(CH * (M + 1) * sizeof(T));
    for (int e = tid; e < nG * CH; e += NT) {
      const int i = e / nG, G = e % nG;
      const bool ok = i < n;
      const void* src = rho_v;   // (a valid address for the zero-filling copies)
      if (ok) {
        const long long p = perm[i0 + i];
        if constexpr (sizeof(T) == 8)
          src = reinterpret_cast<const double2*>(rho_v) + (size_t)G * ld + p;
        else
          src = reinterpret_cast<const float2*>(rho_v) + ((size_t)(p >> 5) * gpad + G) * 32 + (p & 31);
      }
      if constexpr (sizeof(T) == 8)
        cp_async16(rdst + (uint32_t)e * 16u, src, ok ? 16u : 0u);
      else
        cp_async8(rdst + (uint32_t)e * 8u, src, ok ? 8u : 0u);
    }
    for (int e = tid; e < CH * (M + 1); e += NT) {
      const bool ok = e < n * (M + 1);
      const void* src = ok ? (const void*)(coef + (size_t)i0 * (M + 1) + e) : (const void*)coef;
      if constexpr (sizeof(T) == 8)
        cp_async8(cdst + (uint32_t)e * 8u, src, ok ? 8u : 0u);
      else
        cp_async4(cdst + (uint32_t)e * 4u, src, ok ? 4u : 0u);
    }
    if (tid < CH) {
      const bool ok = tid < n;
      cp_async4(bdst + (uint32_t)tid * 4u, ok ? (const void*)(sbin + i0 + tid) : (const void*)sbin,
                ok ? 4u : 0u);
    }
    cp_async_commit();
  };
  if (nchunk > 0) issue(0);
  for (int ck = 0; ck < nchunk; ++ck) {
    const int n = min(CH, rg.y - (rg.x + ck * CH));
    const unsigned char* bufp = sp_smem + (size_t)(ck & 1) * bufsz;
    const T2* rs = reinterpret_cast<const T2*>(bufp);
    const T* cs = reinterpret_cast<const T*>(rs + (size_t)CH * nG);
    const int* bs = reinterpret_cast<const int*>(cs + CH * (M + 1));
    cp_async_wait_all();
    // chunk ck is complete for every thread, and the other buffer's readers (chunk ck - 1) are
    // done
    __syncthreads();
    if (ck + 1 < nchunk) issue(ck + 1);
    for (int i = 0; i < n; ++i) {
      const int j = bs[i];   // the same for every thread
      if (j != cur) {
        flush();
        cur = j;
      }
      T c[M + 1];
#pragma unroll
      for (int k = 0; k <= M; ++k) c[k] = cs[i * (M + 1) + k];
#pragma unroll
      for (int e = 0; e < SP_E; ++e) {
        if (ga[e] < 0) continue;
        const T2 a = rs[i * nG + ga[e]], b = rs[i * nG + gb[e]];
        if constexpr (F32) {
          // a conj(b) = b.x (a.x, a.y) + b.y (a.y, -a.x), and the moments, in packed FP32x2
          const float2 P = __ffma2_rn(make_float2(b.x, b.x), a,
                                      __fmul2_rn(make_float2(b.y, b.y), make_float2(a.y, -a.x)));
#pragma unroll
          for (int k = 0; k <= M; ++k) pp[e][k] = __ffma2_rn(P, make_float2(c[k], c[k]), pp[e][k]);
        } else {
          const T Pr = a.x * b.x + a.y * b.y, Pi = a.y * b.x - a.x * b.y;
#pragma unroll
          for (int k = 0; k <= M; ++k) {
            pp[e][k].x = fma(Pr, c[k], pp[e][k].x);
            pp[e][k].y = fma(Pi, c[k], pp[e][k].y);
          }
        }
      }
    }
    fold();
  }
  flush();
}

// Re A and Im A per G <= G' pair and bin, as the GEMM's left operand: Am [2 ngg][ld]
// (rows Re then Im), A_b = scale sum_c sum_k a[c][k] M_k(j), j = b - c (m = 1) or b + 1 - c (m = 3).
template <typename T, int M>
__global__ void sp_assemble_A(const double2* __restrict__ Mom, int ngg, int nbins, int ld,
                              double scale, T* __restrict__ Am) {
  const long long total = (long long)ngg * nbins;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t % nbins);
    const int g = (int)(t / nbins);
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int c = 0; c <= M; ++c) {
      const int j = (M == 3) ? b + 1 - c : b - c;
      if (j < 0 || j >= nbins) continue;
#pragma unroll
      for (int k = 0; k <= M; ++k) {
        const double a = (M == 3) ? kLag3[c][k] : kLag1[c][k];
        if (a == 0.0) continue;
        const double2 m = Mom[((size_t)j * (M + 1) + k) * ngg + g];
        re += a * m.x;
        im += a * m.y;
      }
    }
    Am[(size_t)g * ld + b] = (T)(scale * re);
    Am[(size_t)(ngg + g) * ld + b] = (T)(scale * im);
  }
}

// Right operand Km [2 ncol][nbins]: rows Re, Im of 1/(w - x_b + i eta) per (eta, w) column.
template <typename T>
__global__ void sp_kernel_matrix(const double* __restrict__ freqs, const double* __restrict__ etas,
                                 int nwi, int ncol, double x0, double h, int nbins,
                                 T* __restrict__ Km) {
  const long long total = (long long)ncol * nbins;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t % nbins);
    const int col = (int)(t / nbins);
    const double w = freqs[col % nwi], eta = etas[col / nwi];
    const double d = w - (x0 + h * b);
    const double r = 1.0 / (d * d + eta * eta);
    Km[(size_t)(2 * col) * nbins + b] = (T)(d * r);
    Km[(size_t)(2 * col + 1) * nbins + b] = (T)(-eta * r);
  }
}

// chi0[col][G][G'] from C [2 ncol][2 ngg] (column-major: C[c * 2 ngg + r]).
template <typename T>
__global__ void sp_unpack(const T* __restrict__ Cm, int ngg, int nG, int ncol, double pref,
                          double2* __restrict__ chi0) {
  const long long total = (long long)ncol * nG * nG;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int Gp = (int)(t % nG);
    const int G = (int)((t / nG) % nG);
    const int col = (int)(t / ((long long)nG * nG));
    const int a = min(G, Gp), b = max(G, Gp);
    const int g = a * nG - a * (a - 1) / 2 + (b - a);
    const size_t ld = 2 * (size_t)ngg;
    const double RR = Cm[(2 * col) * ld + g], RI = Cm[(2 * col + 1) * ld + g];
    const double IR = Cm[(2 * col) * ld + ngg + g], II = Cm[(2 * col + 1) * ld + ngg + g];
    double2 v = (G <= Gp) ? make_double2(RR - II, RI + IR) : make_double2(RR + II, RI - IR);
    chi0[t] = make_double2(pref * v.x, pref * v.y);
  }
}

// Cd = sum over the FP32 partial products of the bin chunks, in FP64.
__global__ void sp_reduce(const float* __restrict__ parts, int nparts, long long n,
                          double* __restrict__ Cd) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < nparts; ++c) acc += (double)parts[(size_t)c * n + i];
    Cd[i] = acc;
  }
}

struct SpState {
  cublasHandle_t blas = nullptr;
  void* buf = nullptr;            // per-pair arrays (x, df, bins, order, coefficients, range)
  size_t bytes = 0;
  void* buf2 = nullptr;           // per-bin arrays (counts, cursors, moments, GEMM operands)
  size_t bytes2 = 0;
  int2* ranges = nullptr;         // block ranges of whole bins
  int ranges_cap = 0;
  std::vector<int2> ranges_h;     // host sources of asynchronous copies, kept alive here
  std::vector<int> start_h;
  double* freqs_etas = nullptr;   // [nwi + neta]
  size_t fe_n = 0;
};

SpState* sp_of(lrt_ctx* c) {
  if (!c->sp) c->sp = new SpState();
  return static_cast<SpState*>(c->sp);
}

size_t al(size_t b) { return (b + 255) / 256 * 256; }

template <typename T, int M>
lrt_status run_spectral(lrt_ctx* c, QData& q, const void* rho, double rho_scale, cudaStream_t s) {
  SpState* S = sp_of(c);
  const int nk = c->nk, nb = c->nb, nG = q.nG;
  const long long np = c->np;
  const int ngg = nG * (nG + 1) / 2;
  const int ncol = lrt::ncol(c);
  const double h = c->spectral_h;
  int dev = 0, nsm = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int grid = 8 * nsm;
  // pass 1: x, df and their range (the grid needs it on the host)
  const size_t b_pairs = al(np * sizeof(double)) * 2 + al(np * sizeof(int)) * 3 +
                         al(np * (M + 1) * sizeof(T)) + al(2 * sizeof(unsigned long long));
  if (S->bytes < b_pairs) {
    cudaFree(S->buf);
    S->buf = nullptr;
    S->bytes = 0;
    LRT_CUDA(cudaMalloc(&S->buf, b_pairs));
    S->bytes = b_pairs;
  }
  char* base = static_cast<char*>(S->buf);
  double* x = reinterpret_cast<double*>(base);
  double* df = reinterpret_cast<double*>(base + al(np * sizeof(double)));
  int* bin = reinterpret_cast<int*>(base + 2 * al(np * sizeof(double)));
  int* perm = reinterpret_cast<int*>(reinterpret_cast<char*>(bin) + al(np * sizeof(int)));
  int* sbin = reinterpret_cast<int*>(reinterpret_cast<char*>(perm) + al(np * sizeof(int)));
  T* coef = reinterpret_cast<T*>(reinterpret_cast<char*>(sbin) + al(np * sizeof(int)));
  unsigned long long* mm =
      reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(coef) + al(np * (M + 1) * sizeof(T)));
  sp_pairs<<<grid, 256, 0, s>>>(q.eps, q.occ, q.wgt, nk, nb, x, df);
  count_launch(c);
  LRT_CUDA(cudaMemsetAsync(mm, 0xff, sizeof(unsigned long long), s));   // min key: all ones
  LRT_CUDA(cudaMemsetAsync(mm + 1, 0, sizeof(unsigned long long), s));  // max key: zero
  sp_range<<<grid, 256, 0, s>>>(x, df, np, mm);
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  unsigned long long hmm[2];
  LRT_CUDA(cudaMemcpyAsync(hmm, mm, sizeof hmm, cudaMemcpyDeviceToHost, s));
  LRT_CUDA(cudaStreamSynchronize(s));
  const size_t chi_bytes = (size_t)ncol * nG * nG * sizeof(double2);
  if (hmm[0] == ~0ull) {   // no pair carries weight: chi0 = 0
    q.sp_x0 = 0.0;
    q.sp_nbins = 0;
    LRT_CUDA(cudaMemsetAsync(q.chi0, 0, chi_bytes, s));
    return LRT_OK;
  }
  // the grid (the oracle's rule): x_0 = h (floor(min x / h) - 1), n_b = floor((max x - x_0)/h) + 3
  const double xmin = ord_val(hmm[0]), xmax = ord_val(hmm[1]);
  const double x0 = h * (std::floor(xmin / h) - 1.0);
  const long long nbl = (long long)std::floor((xmax - x0) / h) + 3;
  if (nbl > (1LL << 26)) {
    set_error("spectral grid too fine for the transition energies (more than 2^26 bins)");
    return LRT_EINVAL;
  }
  const int nbins = (int)nbl;
  q.sp_x0 = x0;
  q.sp_nbins = nbins;
  // second buffer: counts, moments, GEMM operands
  const size_t o_cnt = 0, n_cnt = al((size_t)(nbins + 1) * sizeof(int));
  const size_t o_cur = o_cnt + n_cnt;
  const size_t o_mom = o_cur + n_cnt;
  const size_t n_mom = al((size_t)nbins * (M + 1) * ngg * sizeof(double2));
  // GEMM operands in the moments' type; the split contexts' FP32 transform runs in chunks of
  // SP_KCHUNK bins whose partial products are summed in FP64
  const bool f32 = sizeof(T) == 4;
  const int nbp = f32 ? (nbins + SP_KCHUNK - 1) / SP_KCHUNK * SP_KCHUNK : nbins;
  const int nparts = f32 ? nbp / SP_KCHUNK : 0;
  const long long nC = (long long)2 * ncol * 2 * ngg;
  const size_t o_am = o_mom + n_mom, n_am = al((size_t)2 * ngg * nbp * sizeof(T));
  const size_t o_km = o_am + n_am, n_km = al((size_t)2 * ncol * nbp * sizeof(T));
  const size_t o_c = o_km + n_km, n_c = al((size_t)nC * sizeof(double));
  const size_t o_p = o_c + n_c, n_p = al((size_t)nparts * nC * sizeof(float));
  const size_t need2 = o_p + n_p;
  if (S->bytes2 < need2) {
    cudaFree(S->buf2);
    S->buf2 = nullptr;
    S->bytes2 = 0;
    LRT_CUDA(cudaMalloc(&S->buf2, need2));
    S->bytes2 = need2;
  }
  char* b2 = static_cast<char*>(S->buf2);
  int* count = reinterpret_cast<int*>(b2 + o_cnt);
  int* cursor = reinterpret_cast<int*>(b2 + o_cur);
  double2* Mom = reinterpret_cast<double2*>(b2 + o_mom);
  T* Am = reinterpret_cast<T*>(b2 + o_am);
  T* Km = reinterpret_cast<T*>(b2 + o_km);
  double* Cm = reinterpret_cast<double*>(b2 + o_c);
  float* Cp = reinterpret_cast<float*>(b2 + o_p);
  // pass 2: bins, histogram, exclusive scan (on the host: the block ranges need it there too)
  LRT_CUDA(cudaMemsetAsync(count, 0, (size_t)(nbins + 1) * sizeof(int), s));
  sp_bins<<<grid, 256, 0, s>>>(x, df, np, x0, h, bin, count);
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  std::vector<int> cnt(nbins);
  LRT_CUDA(cudaMemcpyAsync(cnt.data(), count, nbins * sizeof(int), cudaMemcpyDeviceToHost, s));
  LRT_CUDA(cudaStreamSynchronize(s));
  std::vector<int>& start = S->start_h;
  start.assign(nbins + 1, 0);
  for (int j = 0; j < nbins; ++j) start[j + 1] = start[j] + cnt[j];
  const int npos = start[nbins];
  // block ranges of whole bins, about 2048 pairs each (a larger bin is one block)
  std::vector<int2> ranges;
  for (int j = 0; j < nbins;) {
    int j1 = j;
    while (j1 < nbins && (start[j1 + 1] - start[j] < 2048 || j1 == j)) ++j1;
    if (start[j1] > start[j]) ranges.push_back(make_int2(start[j], start[j1]));
    j = j1;
  }
  if (S->ranges_cap < (int)ranges.size()) {
    cudaFree(S->ranges);
    S->ranges = nullptr;
    S->ranges_cap = 0;
    LRT_CUDA(cudaMalloc(&S->ranges, ranges.size() * sizeof(int2)));
    S->ranges_cap = (int)ranges.size();
  }
  S->ranges_h = ranges;   // kept until the copy has run
  LRT_CUDA(cudaMemcpyAsync(S->ranges, S->ranges_h.data(), ranges.size() * sizeof(int2),
                           cudaMemcpyHostToDevice, s));
  LRT_CUDA(cudaMemcpyAsync(cursor, start.data(), nbins * sizeof(int), cudaMemcpyHostToDevice, s));
  sp_scatter<T, M><<<grid, 256, 0, s>>>(x, df, bin, np, x0, h, cursor, perm, sbin, coef);
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  // pass 3: moments per bin (bins without pairs stay zero)
  LRT_CUDA(cudaMemsetAsync(Mom, 0, (size_t)nbins * (M + 1) * ngg * sizeof(double2), s));
  if (npos > 0) {
    // the largest chunk (32, 16 or 8 sorted pairs) whose two buffers fit next to the totals
    constexpr int NT = SpCfg<T>::threads, E = SpCfg<T>::E;
    auto smem_of = [&](int ch) {
      return 2 * ((size_t)nG * ch * sizeof(typename V2<T>::type) + ch * (M + 1) * sizeof(T) +
                  ch * sizeof(int)) +
             (sizeof(T) == 4 ? (size_t)E * (M + 1) * 4 * NT * sizeof(float) : 0);
    };
    const size_t limit = 227 * 1024;
    const int ch = smem_of(32) <= limit ? 32 : (smem_of(16) <= limit ? 16 : 8);
    const size_t smem = smem_of(ch);
    if (smem > limit) {
      set_error("spectral engine: too many G vectors for the moments kernel's shared memory");
      return LRT_EUNSUPPORTED;
    }
    auto kern = ch == 32 ? sp_moments<T, M, 32> : (ch == 16 ? sp_moments<T, M, 16> : sp_moments<T, M, 8>);
    LRT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 g((unsigned)ranges.size(), (unsigned)((ngg + NT * E - 1) / (NT * E)));
    TimedLaunch tl(c, &c->ev_chi0, s);
    kern<<<g, NT, smem, s>>>(rho, c->rho_ld, c->rho_gpad, nG, ngg, perm, sbin, coef,
                                     S->ranges, Mom);
    count_launch(c);
    LRT_CUDA(cudaGetLastError());
  }
  // pass 4: A; 5: the transform GEMM; 6: unpack
  if (nbp > nbins) LRT_CUDA(cudaMemsetAsync(Am, 0, (size_t)2 * ngg * nbp * sizeof(T), s));
  sp_assemble_A<T, M><<<grid, 256, 0, s>>>(Mom, ngg, nbins, nbp, 1.0, Am);
  count_launch(c);
  const size_t nfe = (size_t)c->nwi + c->neta;
  if (S->fe_n < nfe) {
    cudaFree(S->freqs_etas);
    S->freqs_etas = nullptr;
    S->fe_n = 0;
    LRT_CUDA(cudaMalloc(&S->freqs_etas, nfe * sizeof(double)));
    S->fe_n = nfe;
  }
  LRT_CUDA(cudaMemcpyAsync(S->freqs_etas, c->dw.freqs, c->nwi * sizeof(double), cudaMemcpyDeviceToDevice, s));
  LRT_CUDA(cudaMemcpyAsync(S->freqs_etas + c->nwi, c->etas.data(), c->neta * sizeof(double),
                           cudaMemcpyHostToDevice, s));
  LRT_CUDA(cudaStreamSynchronize(s));   // the eta list is read from a host vector
  sp_kernel_matrix<T><<<grid, 256, 0, s>>>(S->freqs_etas, S->freqs_etas + c->nwi, c->nwi, ncol, x0, h,
                                           nbp, Km);
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  if (!S->blas && cublasCreate(&S->blas) != CUBLAS_STATUS_SUCCESS) {
    set_error("cublasCreate failed");
    return LRT_ECUDA;
  }
  cublasSetStream(S->blas, s);
  // The sum over all bins cancels between the bins below and above each frequency: one FP32
  // accumulation over ~10^4 bins loses ~1e-5 of the result to it, so the FP32 products are
  // accumulated over SP_KCHUNK bins at a time and the chunks summed in FP64 (FP64 context:
  // one DGEMM).
  cublasStatus_t st;
  if constexpr (sizeof(T) == 4) {
    const float one = 1.f, zero = 0.f;
    st = cublasSgemmStridedBatched(S->blas, CUBLAS_OP_T, CUBLAS_OP_N, 2 * ngg, 2 * ncol, SP_KCHUNK,
                                   &one, Am, nbp, SP_KCHUNK, Km, nbp, SP_KCHUNK, &zero, Cp, 2 * ngg,
                                   nC, nparts);
    if (st == CUBLAS_STATUS_SUCCESS) {
      sp_reduce<<<grid, 256, 0, s>>>(Cp, nparts, nC, Cm);
      count_launch(c);
    }
  } else {
    const double one = 1, zero = 0;
    st = cublasDgemm(S->blas, CUBLAS_OP_T, CUBLAS_OP_N, 2 * ngg, 2 * ncol, nbins, &one, Am, nbins, Km,
                     nbins, &zero, Cm, 2 * ngg);
  }
  if (st != CUBLAS_STATUS_SUCCESS) {
    set_error("spectral transform GEMM failed");
    return LRT_ECUDA;
  }
  const double pref = 2.0 / (c->nk * c->volume) / (rho_scale * rho_scale);
  sp_unpack<double><<<grid, 256, 0, s>>>(Cm, ngg, nG, ncol, pref, q.chi0);
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  return LRT_OK;
}

}  // namespace

lrt_status launch_chi0_spectral(lrt_ctx* c, QData& q, const void* rho, cudaStream_t s) {
  const bool fp64 = c->precision == LRT_PREC_FP64;
  const double rs = fp64 ? 1.0 : (double)split_rho_scale(c->precision);
  if (fp64)
    return c->spectral_order == 3 ? run_spectral<double, 3>(c, q, rho, rs, s)
                                  : run_spectral<double, 1>(c, q, rho, rs, s);
  return c->spectral_order == 3 ? run_spectral<float, 3>(c, q, rho, rs, s)
                                : run_spectral<float, 1>(c, q, rho, rs, s);
}

void free_spectral_state(lrt_ctx* c) {
  if (!c->sp) return;
  SpState* S = static_cast<SpState*>(c->sp);
  if (S->blas) cublasDestroy(S->blas);
  cudaFree(S->buf);
  cudaFree(S->buf2);
  cudaFree(S->ranges);
  cudaFree(S->freqs_etas);
  delete S;
  c->sp = nullptr;
}

}  // namespace lrt
