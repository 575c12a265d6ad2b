// The eta-convergence test and the attenuation started from the Kubo-Greenwood conductivity
// (App. A.3), in the optical limit q -> 0 of the interband response, on the k mesh (and the
// orbitals) of q index 0 of the context, FP64 throughout:
//   p_nn'(k)    = <nk| -i grad |n'k> = sum_G c*_nk(G) (k + G) c_n'k(G)           (momentum)
//   L(w)        = (2/(N_k Omega)) sum_{k,n,n'} df_nn' (|p_nn'|^2/3) / Delta^2 / (w + Delta + i eta),
//                 Delta = eps_nk - eps_n'k, df_nn' = w_nk w_n'k (f_nk - f_n'k), pairs with
//                 Delta = 0 left out (their df is 0): L = lim chi0_inter(q, w)/q^2, trace/3
//   sigma_KG(w) = i w L(w),   eps_KG = 1 + 4 pi i sigma_KG/w = 1 - 4 pi L      (Eq. 11)
//   chi*_KG     = 1/eps_KG - 1                                       (Eqs. 10 and 12, v chi)
//   S*_KG(w)    = -Im chi*_KG / (pi n (1 - e^{-w/T})),                       (Eq. 13)
//   S*_KG(0)    = (T/(pi n)) Re[4 pi L_eta(0) / eps_KG(0)^2],  L_eta = dL/d eta (L depends on
//                 w + i eta only, the same limit as S(q,0))
// then F*_KG (Eq. 14) and the Sec. 2 metrics by the fold of Eq. 1, the reference eta (Sec. 2), and, for
// the reference eta, the attenuation of S*_KG and the filtered chi*, eps and sigma
// (Kramers-Kronig, Eqs. 10-11 with v = 1).
#include <algorithm>
#include <cmath>
#include <vector>

#include "lrt_internal.h"

namespace lrt {

struct KgState {
  double* S = nullptr;       // [n_eta][nw] S*_KG of the last scan
  double2* s0 = nullptr;     // [n_eta] 4 pi L_eta(0)/eps(0)^2  (S*(0) = T Re s0/(pi n))
  int neta = 0;
  int ref = -1;              // reference eta of the last scan
};

void free_kg_state(lrt_ctx* c) {
  if (!c->kg) return;
  KgState* K = static_cast<KgState*>(c->kg);
  cudaFree(K->S);
  cudaFree(K->s0);
  delete K;
  c->kg = nullptr;
}

namespace {

__device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

constexpr int KT = 32;   // n and n' per tile
constexpr int KG = 16;   // plane waves per step

// Pair weights of the optical limit: grid (n tile, n' tile, k); 256 threads, 4 outputs each.
// delta[p], g[p] for p = (k nb + n) nb + n'.
__global__ void __launch_bounds__(256) kg_pairs_kernel(
    const double2* __restrict__ coeff, const double* __restrict__ kg, const double* __restrict__ eps,
    const double* __restrict__ occ, const double* __restrict__ wgt, int nk, int nb, int npw,
    double pref, double* __restrict__ delta, double* __restrict__ g) {
  __shared__ double2 A[KG][KT];
  __shared__ double2 B[KG][KT];
  __shared__ double P[KG][3];
  const int ntile = (nb + KT - 1) / KT;
  const int tn = blockIdx.x / ntile, tm = blockIdx.x % ntile, k = blockIdx.y;
  const int tid = threadIdx.x;
  const int lm = tid & 31, ln = tid >> 5;    // this thread: n' = tm KT + lm, n = tn KT + ln + 8 i
  double2 acc[4][3];
  for (int i = 0; i < 4; ++i)
    for (int a = 0; a < 3; ++a) acc[i][a] = make_double2(0.0, 0.0);
  const double2* Ck = coeff + (size_t)k * nb * npw;
  for (int g0 = 0; g0 < npw; g0 += KG) {
    for (int e = tid; e < KG * KT; e += 256) {
      const int gg = e / KT, t = e % KT;
      const int G = g0 + gg, n1 = tn * KT + t, n2 = tm * KT + t;
      A[gg][t] = (G < npw && n1 < nb) ? Ck[(size_t)n1 * npw + G] : make_double2(0.0, 0.0);
      B[gg][t] = (G < npw && n2 < nb) ? Ck[(size_t)n2 * npw + G] : make_double2(0.0, 0.0);
    }
    if (tid < KG * 3) {
      const int gg = tid / 3, a = tid % 3, G = g0 + gg;
      P[gg][a] = G < npw ? kg[((size_t)k * npw + G) * 3 + a] : 0.0;
    }
    __syncthreads();
    for (int gg = 0; gg < KG; ++gg) {
      const double2 b = B[gg][lm];
      for (int i = 0; i < 4; ++i) {
        const double2 a = A[gg][ln + 8 * i];
        // conj(a) b
        const double2 ab = make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
        for (int c = 0; c < 3; ++c) {
          acc[i][c].x += P[gg][c] * ab.x;
          acc[i][c].y += P[gg][c] * ab.y;
        }
      }
    }
    __syncthreads();
  }
  const int m = tm * KT + lm;
  if (m >= nb) return;
  for (int i = 0; i < 4; ++i) {
    const int n = tn * KT + ln + 8 * i;
    if (n >= nb) continue;
    double p2 = 0.0;
    for (int c = 0; c < 3; ++c) p2 += acc[i][c].x * acc[i][c].x + acc[i][c].y * acc[i][c].y;
    const size_t a1 = (size_t)k * nb + n, a2 = (size_t)k * nb + m;
    const double d = eps[a1] - eps[a2];
    const double df = wgt[a1] * wgt[a2] * (occ[a1] - occ[a2]);
    const size_t p = ((size_t)k * nb + n) * nb + m;
    delta[p] = d;
    g[p] = d != 0.0 ? pref * df * p2 / (3.0 * d * d) : 0.0;
  }
}

// L[e][col] += sum over this block's pairs of g/(f_col + Delta + i eta_e) for col < nw + 1
// (f_col = omega[col], f_nw = 0) and -i g/(Delta + i eta_e)^2 for col = nw + 1.
// grid (column tiles of 256, eta, pair splits); thread = column.
__global__ void __launch_bounds__(256) kg_sum_kernel(const double* __restrict__ delta,
                                                     const double* __restrict__ g,
                                                     const double* __restrict__ omega, int nw,
                                                     const double* __restrict__ etas, long long np,
                                                     long long per, double2* __restrict__ L) {
  __shared__ double ds[256], gs[256];
  const int col = blockIdx.x * 256 + threadIdx.x;
  const int ncol = nw + 2;
  const double eta = etas[blockIdx.y];
  const double f = col < nw ? omega[col] : 0.0;
  const long long pb = (long long)blockIdx.z * per, pe = min(np, pb + per);
  double sr = 0.0, si = 0.0;
  for (long long p0 = pb; p0 < pe; p0 += 256) {
    __syncthreads();
    const long long p = p0 + threadIdx.x;
    ds[threadIdx.x] = p < pe ? delta[p] : 0.0;
    gs[threadIdx.x] = p < pe ? g[p] : 0.0;
    __syncthreads();
    if (col >= ncol) continue;
    const int cnt = (int)min((long long)256, pe - p0);
    if (col <= nw) {
      for (int j = 0; j < cnt; ++j) {
        const double x = f + ds[j], den = x * x + eta * eta;
        const double s = gs[j] / den;
        sr += s * x;
        si -= s * eta;
      }
    } else {
      for (int j = 0; j < cnt; ++j) {
        // -i g / (Delta + i eta)^2 = g (-2 Delta eta - i (Delta^2 - eta^2)) / |Delta + i eta|^4
        const double x = ds[j], den = x * x + eta * eta;
        const double s = gs[j] / (den * den);
        sr += -2.0 * s * x * eta;
        si += -s * (x * x - eta * eta);
      }
    }
  }
  if (col < ncol) {
    atomicAdd(&L[(size_t)blockIdx.y * ncol + col].x, sr);
    atomicAdd(&L[(size_t)blockIdx.y * ncol + col].y, si);
  }
}

// sigma, S*_KG and s0 per eta from L [n_eta][nw + 2].
__global__ void kg_post_kernel(const double2* __restrict__ L, const double* __restrict__ omega, int nw,
                               int neta, double T, double n, double2* __restrict__ sigma,
                               double* __restrict__ S, double2* __restrict__ s0) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= neta * (nw + 1)) return;
  const int e = t / (nw + 1), j = t % (nw + 1);
  const double2* Le = L + (size_t)e * (nw + 2);
  if (j == nw) {   // w = 0: s0 = 4 pi L_eta(0) / eps(0)^2
    const double2 e0 = make_double2(1.0 - 4.0 * M_PI * Le[nw].x, -4.0 * M_PI * Le[nw].y);
    const double2 e2 = cmul(e0, e0);
    const double d = e2.x * e2.x + e2.y * e2.y;
    const double2 num = make_double2(4.0 * M_PI * Le[nw + 1].x, 4.0 * M_PI * Le[nw + 1].y);
    s0[e] = make_double2((num.x * e2.x + num.y * e2.y) / d, (num.y * e2.x - num.x * e2.y) / d);
    return;
  }
  const double w = omega[j];
  const double2 l = Le[j];
  sigma[(size_t)e * nw + j] = make_double2(-w * l.y, w * l.x);   // i w L
  // chi* = 1/eps - 1, eps = 1 - 4 pi L;  Im(1/eps) = -Im(eps)/|eps|^2
  const double er = 1.0 - 4.0 * M_PI * l.x, ei = -4.0 * M_PI * l.y;
  const double im = -ei / (er * er + ei * ei);
  double v;
  if (w == 0.0) {
    const double2 e0 = make_double2(er, ei);
    const double2 e2 = cmul(e0, e0);
    const double d = e2.x * e2.x + e2.y * e2.y;
    const double2 num = make_double2(4.0 * M_PI * Le[nw + 1].x, 4.0 * M_PI * Le[nw + 1].y);
    v = T * ((num.x * e2.x + num.y * e2.y) / d) / (M_PI * n);
  } else {
    v = -im / (M_PI * n * (-expm1(-w / T)));
  }
  S[(size_t)e * nw + j] = v;
}

}  // namespace
}  // namespace lrt

using namespace lrt;

extern "C" lrt_status lrtddft_kubo_greenwood(lrt_ctx* c, int n_eta, const double* eta, int ntau,
                                             const double* tau, double tol, double* sigma, double* S,
                                             double* F, double* metrics, int* eta_ref) {
  if (!c || !eta || !tau || !eta_ref) {
    set_error("NULL argument");
    return LRT_EINVAL;
  }
  if (c->host_only) {
    set_error("host-only context");
    return LRT_ESTATE;
  }
  if (n_eta < 1 || n_eta > 64) {
    set_error("n_eta must be in 1..64");
    return LRT_EINVAL;
  }
  for (int j = 0; j < n_eta; ++j)
    if (!(eta[j] > 0) || !std::isfinite(eta[j]) || (j > 0 && !(eta[j] > eta[j - 1]))) {
      set_error("etas must be positive, finite and strictly increasing");
      return LRT_EINVAL;
    }
  if (!(tol >= 0) || !std::isfinite(tol)) {
    set_error("tol must be finite and >= 0");
    return LRT_EINVAL;
  }
  if (ntau < 1) {
    set_error("ntau must be >= 1");
    return LRT_EINVAL;
  }
  for (int i = 0; i < ntau; ++i)
    if (!(tau[i] >= 0.0) || tau[i] > 1.0 / c->T * (1.0 + 1e-12)) {
      set_error("tau outside [0, beta]");
      return LRT_EINVAL;
    }
  LRT_CUDA(cudaSetDevice(c->device));
  LRT_TRY(adopt_orbitals(c, 0, 0));
  LRT_CUDA(cudaDeviceSynchronize());
  const QData& Q = c->qd[0];
  const int nk = c->nk, nb = c->nb, npw = c->npw, nw = c->nw;
  const long long np = (long long)nk * nb * nb;
  // (k + G) of the k mesh of q 0, padding rows zero
  std::vector<double> kg((size_t)nk * npw * 3, 0.0);
  for (int k = 0; k < nk; ++k)
    for (int G = 0; G < Q.npw_k[k]; ++G) {
      const int32_t* mi = &Q.miller[((size_t)k * npw + G) * 3];
      for (int a = 0; a < 3; ++a)
        kg[((size_t)k * npw + G) * 3 + a] = Q.kpts[3 * k + a] + mi[0] * c->recip[0][a] +
                                            mi[1] * c->recip[1][a] + mi[2] * c->recip[2][a];
    }
  if (!c->kg) c->kg = new KgState();
  KgState* K = static_cast<KgState*>(c->kg);
  if (K->neta != n_eta) {
    cudaFree(K->S);
    cudaFree(K->s0);
    K->S = nullptr;
    K->s0 = nullptr;
    K->neta = 0;
    LRT_CUDA(cudaMalloc(&K->S, (size_t)n_eta * nw * sizeof(double)));
    LRT_CUDA(cudaMalloc(&K->s0, (size_t)n_eta * sizeof(double2)));
    K->neta = n_eta;
  }
  K->ref = -1;
  double *d_kg = nullptr, *d_delta = nullptr, *d_g = nullptr, *d_eta = nullptr, *d_tau = nullptr,
         *d_F = nullptr, *d_m = nullptr;
  double2 *d_L = nullptr, *d_sigma = nullptr;
  int* d_ref = nullptr;
  auto done = [&](lrt_status st) {
    cudaFree(d_kg);
    cudaFree(d_delta);
    cudaFree(d_g);
    cudaFree(d_eta);
    cudaFree(d_tau);
    cudaFree(d_F);
    cudaFree(d_m);
    cudaFree(d_L);
    cudaFree(d_sigma);
    cudaFree(d_ref);
    return st;
  };
  const int ncol = nw + 2;
  if (cudaMalloc(&d_kg, kg.size() * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_delta, np * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_g, np * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_eta, n_eta * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_tau, ntau * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_F, (size_t)n_eta * ntau * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_m, (size_t)n_eta * 5 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_L, (size_t)n_eta * ncol * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&d_sigma, (size_t)n_eta * nw * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&d_ref, sizeof(int)) != cudaSuccess) {
    set_error("device allocation");
    return done(LRT_ENOMEM);
  }
  if (cudaMemcpy(d_kg, kg.data(), kg.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_eta, eta, n_eta * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_tau, tau, ntau * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(d_L, 0, (size_t)n_eta * ncol * sizeof(double2)) != cudaSuccess)
    return done(LRT_ECUDA);
  const int ntile = (nb + KT - 1) / KT;
  const double pref = 2.0 / (nk * c->volume);
  kg_pairs_kernel<<<dim3(ntile * ntile, nk), 256>>>(Q.coeff, d_kg, Q.eps, Q.occ, Q.wgt, nk, nb, npw, pref,
                                                    d_delta, d_g);
  int dev = 0, nsm = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int ntile_c = (ncol + 255) / 256;
  long long nz = std::max<long long>(1, (4LL * nsm + (long long)ntile_c * n_eta - 1) / ((long long)ntile_c * n_eta));
  long long per = (np + nz - 1) / nz;
  per = (per + 255) / 256 * 256;
  nz = (np + per - 1) / per;
  kg_sum_kernel<<<dim3(ntile_c, n_eta, (unsigned)nz), 256>>>(d_delta, d_g, c->dw.omega, nw, d_eta, np,
                                                            per, d_L);
  kg_post_kernel<<<(n_eta * (nw + 1) + 255) / 256, 256>>>(d_L, c->dw.omega, nw, n_eta, c->T, c->density,
                                                          d_sigma, K->S, K->s0);
  count_launch(c, 3);
  if (cudaGetLastError() != cudaSuccess) return done(LRT_ECUDA);
  lrt_status st = launch_itcf_rows(c, K->S, K->s0, n_eta, ntau, d_tau, LRT_ITCF_FOLD, d_F, d_m, 0);
  if (st == LRT_OK) st = launch_eta_pick(c, d_m, 1, n_eta, tol, d_ref, 0);
  if (st != LRT_OK) return done(st);
  if ((sigma && cudaMemcpy(sigma, d_sigma, (size_t)n_eta * nw * sizeof(double2), cudaMemcpyDeviceToHost) !=
                    cudaSuccess) ||
      (S && cudaMemcpy(S, K->S, (size_t)n_eta * nw * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (F && cudaMemcpy(F, d_F, (size_t)n_eta * ntau * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (metrics && cudaMemcpy(metrics, d_m, (size_t)n_eta * 5 * sizeof(double), cudaMemcpyDeviceToHost) !=
                      cudaSuccess) ||
      cudaMemcpy(eta_ref, d_ref, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return done(LRT_ECUDA);
  K->ref = *eta_ref;
  return done(LRT_OK);
}

extern "C" lrt_status lrtddft_kubo_greenwood_attenuate(lrt_ctx* c, const lrt_atten_params* p, double* Sp,
                                                       lrt_atten_report* rep, double* out) {
  if (!c || !Sp) {
    set_error("NULL argument");
    return LRT_EINVAL;
  }
  KgState* K = static_cast<KgState*>(c->kg);
  if (!K || K->ref < 0) {
    set_error("kubo_greenwood_attenuate before a kubo_greenwood scan");
    return LRT_ESTATE;
  }
  LRT_CUDA(cudaSetDevice(c->device));
  LRT_CUDA(cudaDeviceSynchronize());
  LRT_TRY(run_attenuation_rows(c, p, K->S + (size_t)K->ref * c->nw, K->s0 + K->ref, 1, Sp, rep, 0));
  if (out) {
    const double one = 1.0;   // chi* already carries v(q)
    LRT_TRY(run_dielectric(c, Sp, 1, &one, out));
  }
  return check_status_word(c);
}
