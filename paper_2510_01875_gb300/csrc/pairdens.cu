// Pair densities rho_p(G) = <nk| e^{-i(q+G).r} |n'k+q> = sum_G1 c*_nk(G1) c_n'k+q(G1+G)
// as a G-space correlation: for each (k, G) a complex GEMM over the plane-wave index with the
// k+q operand gathered through a precomputed index table (G1 + G -> position in the k+q
// basis).  This costs N_pw N_G complex MACs per pair, against N_r log N_r for the same
// coefficients taken from an FFT of u*_nk u_n'k+q on the real-space grid (N_pw N_G is
// 15-50x smaller at these cut-offs).
//
// Output layout, p = (k nb + n) nb + n':
//  FP64 path: rho[G][p] with row stride ld (the pair count rounded up to 32);
//  split path: blocked rho[p / 32][G][p % 32] with G padded to a multiple of 8, so that the rows
//  of one 8-G block for one 32-pair stage are a single contiguous 2 KB copy; the values carry
//  the exact power-of-two factor split_rho_scale().
#include "lrt_internal.h"

namespace lrt {
namespace {

template <typename R>
struct C2;
template <>
struct C2<double> {
  using T = double2;
};
template <>
struct C2<float> {
  using T = float2;
};

constexpr int TN = 64;   // n and n' tile
constexpr int TK = 16;   // plane waves per step

// grid: x = (n tile, n' tile), y = G, z = k.  256 threads; each owns 4 x 4 outputs.
template <typename R>
__global__ void __launch_bounds__(256) pair_density_kernel(
    const double2* __restrict__ ck, const double2* __restrict__ ckq,
    const int32_t* __restrict__ gather, int nk, int nb, int npw, int nG, int ntile, int64_t ld,
    int nGpad, R scale, typename C2<R>::T* __restrict__ rho) {
  using CT = typename C2<R>::T;
  __shared__ CT As[TK][TN];
  __shared__ CT Bs[TK][TN];
  const int k = blockIdx.z;
  const int G = blockIdx.y;
  const int n0 = (blockIdx.x / ntile) * TN;
  const int m0 = (blockIdx.x % ntile) * TN;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const double2* A = ck + (size_t)k * nb * npw;
  const double2* B = ckq + (size_t)k * nb * npw;
  const int32_t* tab = gather + ((size_t)k * nG + G) * npw;
  R accr[4][4], acci[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = R(0);
  for (int g0 = 0; g0 < npw; g0 += TK) {
    // 1024 elements of each operand per step, 4 per thread, g fastest
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + 256 * r;
      int g = e % TK, n = e / TK;
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
      if (g0 + g < npw) {
        if (n0 + n < nb) a = A[(size_t)(n0 + n) * npw + g0 + g];
        int j = tab[g0 + g];
        if (j >= 0 && m0 + n < nb) b = B[(size_t)(m0 + n) * npw + j];
      }
      As[g][n] = CT{(R)a.x, (R)a.y};
      Bs[g][n] = CT{(R)b.x, (R)b.y};
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < TK; ++g) {
      CT a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[g][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[g][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          // conj(a) * b
          accr[i][j] += a[i].x * b[j].x + a[i].y * b[j].y;
          acci[i][j] += a[i].x * b[j].y - a[i].y * b[j].x;
        }
    }
    __syncthreads();
  }
  const int64_t kbase = (int64_t)k * nb * nb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int n = n0 + ty + 16 * i;
    if (n >= nb) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int m = m0 + tx + 16 * j;
      if (m >= nb) continue;
      const int64_t p = kbase + (int64_t)n * nb + m;
      // row layout rho[G][p] (nGpad == 0) or blocked rho[p / 32][G][p % 32]
      const size_t idx = nGpad ? ((size_t)((p >> 5) * nGpad + G) << 5) + (size_t)(p & 31)
                               : (size_t)G * ld + (size_t)p;
      rho[idx] = CT{accr[i][j] * scale, acci[i][j] * scale};
    }
  }
}

// Delta_p = eps_nk - eps_n'k+q and df_p = w_nk w_n'k+q (f_nk - f_n'k+q) (band weights w).
__global__ void pair_weights_kernel(const double* __restrict__ eps, const double* __restrict__ occ,
                                    const double* __restrict__ wgt, int nk, int nb,
                                    double* __restrict__ delta, double* __restrict__ df) {
  int64_t np = (int64_t)nk * nb * nb;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x) {
    int m = (int)(p % nb);
    int64_t kn = p / nb;  // k nb + n
    int k = (int)(kn / nb);
    size_t ikq = (size_t)(nk + k) * nb + m;
    delta[p] = eps[kn] - eps[ikq];
    df[p] = wgt[kn] * wgt[ikq] * (occ[kn] - occ[ikq]);
  }
}

}  // namespace

lrt_status launch_pair_density(const lrt_ctx* c, const QData& q, void* rho, bool fp32,
                               cudaStream_t s) {
  // split path: tensor cores unless the caller asked for this kernel
  if (fp32 && !c->pair_simt) return launch_pair_density_tc(c, q, rho, s);
  int ntile = (c->nb + TN - 1) / TN;
  dim3 grid(ntile * ntile, q.nG, c->nk);
  const double2* ck = q.coeff;
  const double2* ckq = q.coeff + (size_t)c->nk * c->nb * c->npw;
  {
    TimedLaunch tl(c, &c->ev_rho, s);
    if (fp32)
      pair_density_kernel<float><<<grid, 256, 0, s>>>(ck, ckq, q.gather, c->nk, c->nb, c->npw, q.nG,
                                                      ntile, c->rho_ld, c->rho_gpad,
                                                      split_rho_scale(c->precision), (float2*)rho);
    else
      pair_density_kernel<double><<<grid, 256, 0, s>>>(ck, ckq, q.gather, c->nk, c->nb, c->npw,
                                                       q.nG, ntile, c->rho_ld, 0, 1.0, (double2*)rho);
  }
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  return LRT_OK;
}

lrt_status launch_pair_weights(const lrt_ctx* c, const QData& q, cudaStream_t s) {
  pair_weights_kernel<<<1216, 256, 0, s>>>(q.eps, q.occ, q.wgt, c->nk, c->nb, c->dw.delta, c->dw.df);
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  return LRT_OK;
}

}  // namespace lrt
