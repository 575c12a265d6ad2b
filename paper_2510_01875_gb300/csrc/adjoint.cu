// Tangents of chi_00(q, w) with respect to theta = (T, eta, A, B, C): the part of the adjoint
// of S(q, w) (Eq. 8) and F(q, tau) (Eq. 1) that touches the response functions.
//
// With M = 1 - chi0 K (K diagonal), chi_{:,0} = M^{-1} chi0_{:,0} and a change d of chi0 and K,
//   d chi_00 = u^T d chi0 v + u^T chi0 dK chi_{:,0},   M^T u = e_0,   v = K chi_{:,0} + e_0.
// The Dyson LU is recomputed from the stored chi0 (one block per frequency, Mᵀ u = e_0 by
// Gaussian elimination with partial pivoting; Mᵀ in shared memory up to N_G = 118, above that
// in a per-block slice of a global workspace), which also gives the f_xc-model terms
// u^T chi0 dK chi_{:,0} for A, B, C.  The T and eta terms need the weight tangents inside the
// pair sum:
//   u^T d chi0 v = (2/(N_k Omega)) sum_p a_p(w) b_p(w) dw_p(w),
//   a_p(w) = sum_G u_G(w) rho_p(G),   b_p(w) = sum_G' rho_p*(G') v_G'(w),
//   dw_p/dT = (d df_p/dT)/(w + Delta_p + i eta),   dw_p/deta = -i df_p/(w + Delta_p + i eta)^2,
//   d df_p/dT = w_nk w_n'k+q (df_nk/dT - df_n'k+q/dT),
//   df/dT = f (1 - f) ((eps - mu)/T^2 + mu'/T),  mu' from the conserved electron count.
// The projections are computed for every (p, w) on the fly from the pair densities (2 N_G
// complex MACs each) and reduced over p; nothing of size N_p x N_w is stored.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lrt_internal.h"

namespace lrt {
namespace {

__device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ inline double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// Block loop over frequencies w = blockIdx.x, blockIdx.x + gridDim.x, ...  GM: M^T in ws
// (N x (N+1) per block) and shared memory rhs[N], fac[N]; otherwise shared memory N x (N+1)
// matrix M^T, then rhs[N], fac[N].  Outputs per frequency: u[N], v[N] and the A, B, C tangents
// of chi_00 (dK holds the three tangents of the kernel diagonal, [3][N]).
template <bool GM>
__global__ void __launch_bounds__(256) dyson_adjoint_kernel(
    const double2* __restrict__ chi0, const double* __restrict__ K, const double* __restrict__ dK,
    const double2* __restrict__ chi, int N, int nw, double2* __restrict__ u_out,
    double2* __restrict__ v_out, double2* __restrict__ dk_out, int* __restrict__ status,
    double2* ws) {
  extern __shared__ double2 sm[];
  const int ld = N + 1;
  double2* A = GM ? ws + (size_t)blockIdx.x * N * ld : sm;
  double2* b = GM ? sm : sm + (size_t)N * ld;
  double2* fac = b + N;
  __shared__ int piv_s;
  __shared__ int bad;
  __shared__ double2 red_s[8];   // per-warp partials (256 threads)
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) bad = 0;
  for (int w = blockIdx.x; w < nw; w += gridDim.x) {
    const double2* X = chi0 + (size_t)w * N * N;
    const double2* x = chi + (size_t)w * N;
    __syncthreads();   // the previous frequency is done with A, b and fac
    // A = M^T: A[r][j] = M[j][r] = delta_jr - chi0[j][r] K[r]
    for (int e = tid; e < N * N; e += nt) {
      int j = e / N, r = e % N;
      double2 v = X[e];
      double2 m = make_double2(-v.x * K[r], -v.y * K[r]);
      if (r == j) m.x += 1.0;
      A[r * ld + j] = m;
    }
    for (int r = tid; r < N; r += nt) b[r] = make_double2(r == 0 ? 1.0 : 0.0, 0.0);
    __syncthreads();
    for (int c = 0; c < N; ++c) {
      if (tid < 32) {
        double best = -1.0;
        int bi = c;
        for (int r = c + tid; r < N; r += 32) {
          double2 v = A[r * ld + c];
          double a = v.x * v.x + v.y * v.y;
          if (a > best) {
            best = a;
            bi = r;
          }
        }
        for (int off = 16; off > 0; off >>= 1) {
          double ob = __shfl_down_sync(0xffffffffu, best, off);
          int oi = __shfl_down_sync(0xffffffffu, bi, off);
          if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
          }
        }
        if (tid == 0) {
          piv_s = bi;
          if (!(best > 0.0)) bad = 1;
        }
      }
      __syncthreads();
      const int p = piv_s;
      if (p != c) {
        for (int j = tid; j < N; j += nt) {
          double2 t = A[c * ld + j];
          A[c * ld + j] = A[p * ld + j];
          A[p * ld + j] = t;
        }
        if (tid == 0) {
          double2 t = b[c];
          b[c] = b[p];
          b[p] = t;
        }
      }
      __syncthreads();
      const double2 d = A[c * ld + c];
      for (int r = c + 1 + tid; r < N; r += nt) fac[r] = cdiv(A[r * ld + c], d);
      __syncthreads();
      const int rows = N - c - 1, cols = N - c;
      for (int e = tid; e < rows * cols; e += nt) {
        int r = c + 1 + e / cols;
        int jj = e % cols;
        double2 f = fac[r];
        if (jj == cols - 1) {
          double2 t = cmul(f, b[c]);
          b[r].x -= t.x;
          b[r].y -= t.y;
        } else {
          int j = c + 1 + jj;
          double2 t = cmul(f, A[c * ld + j]);
          A[r * ld + j].x -= t.x;
          A[r * ld + j].y -= t.y;
        }
      }
      __syncthreads();
    }
    for (int c = N - 1; c >= 0; --c) {
      if (tid == 0) b[c] = cdiv(b[c], A[c * ld + c]);
      __syncthreads();
      const double2 xc = b[c];
      for (int r = tid; r < c; r += nt) {
        double2 t = cmul(A[r * ld + c], xc);
        b[r].x -= t.x;
        b[r].y -= t.y;
      }
      __syncthreads();
    }
    // u = b.  v = K x + e_0.  r_G' = sum_G u_G chi0[G][G'];  dchi_00/dtheta_j = sum_G' r_G' dK_j,G' x_G'
    for (int r = tid; r < N; r += nt) {
      u_out[(size_t)w * N + r] = b[r];
      double2 xv = x[r];
      v_out[(size_t)w * N + r] = make_double2(K[r] * xv.x + (r == 0 ? 1.0 : 0.0), K[r] * xv.y);
    }
    double2 acc[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    for (int gp = tid; gp < N; gp += nt) {
      double2 rg = make_double2(0, 0);
      for (int g = 0; g < N; ++g) {
        double2 t = cmul(b[g], X[(size_t)g * N + gp]);
        rg.x += t.x;
        rg.y += t.y;
      }
      const double2 rx = cmul(rg, x[gp]);
      for (int j = 0; j < 3; ++j) {
        acc[j].x += rx.x * dK[j * N + gp];
        acc[j].y += rx.y * dK[j * N + gp];
      }
    }
    // block reduction of the three sums (one partial per warp)
    for (int j = 0; j < 3; ++j) {
      double2 v = acc[j];
      for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, off);
        v.y += __shfl_down_sync(0xffffffffu, v.y, off);
      }
      __syncthreads();
      if ((tid & 31) == 0) red_s[tid >> 5] = v;
      __syncthreads();
      if (tid == 0) {
        double2 s = make_double2(0, 0);
        for (int i = 0; i < (nt >> 5); ++i) {
          s.x += red_s[i].x;
          s.y += red_s[i].y;
        }
        dk_out[(size_t)w * 3 + j] = s;
      }
    }
  }
  if (tid == 0 && bad) atomicOr(status, 1);
}

// Per pair: Delta_p, df_p and d df_p/dT (all FP64).
__global__ void adjoint_pair_weights(const double* __restrict__ eps, const double* __restrict__ occ,
                                     const double* __restrict__ wgt, int nk, int nb, double mu,
                                     double T, double mup, int fixed, double* __restrict__ delta,
                                     double* __restrict__ df, double* __restrict__ ddf) {
  long long np = (long long)nk * nb * nb;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    int m = (int)(p % nb);
    long long kn = p / nb;
    int k = (int)(kn / nb);
    size_t ikq = (size_t)(nk + k) * nb + m;
    const double w = wgt[kn] * wgt[ikq];
    delta[p] = eps[kn] - eps[ikq];
    df[p] = w * (occ[kn] - occ[ikq]);
    double d = 0.0;
    if (!fixed) {
      const double f1 = occ[kn], f2 = occ[ikq];
      const double t1 = f1 * (1.0 - f1) * ((eps[kn] - mu) / (T * T) + mup / T);
      const double t2 = f2 * (1.0 - f2) * ((eps[ikq] - mu) / (T * T) + mup / T);
      d = w * (t1 - t2);
    }
    ddf[p] = d;
  }
}

template <typename R>
struct CT;
template <>
struct CT<float> {
  using T2 = float2;
};
template <>
struct CT<double> {
  using T2 = double2;
};

constexpr int PCH = 32;    // pairs per chunk (one per lane)
constexpr int OG = 8;      // frequency groups (warps) per block
constexpr size_t kProjSmem = 200 * 1024;   // shared-memory budget of the projection tiles

// Projections and the pair sum for the T and eta tangents.
// grid: x = pair split, y = frequency tile of WT.  Block: 256 threads = 8 warps; lane = pair of
// the chunk, warp = group of WT/8 frequencies.  g[w] gets {Re, Im} of sum_p a b ddf/den and of
// sum_p a b (-i df)/den^2 (den = w + Delta + i eta), in the units of rho^2.
template <typename R, int WT>
__global__ void __launch_bounds__(256) adjoint_project_kernel(
    const typename CT<R>::T2* __restrict__ rho, long long ld, int gpad, int nG,
    const double2* __restrict__ u, const double2* __restrict__ v, const double* __restrict__ freqs,
    int nwi, const double* __restrict__ delta, const double* __restrict__ df,
    const double* __restrict__ ddf, long long np, long long per_split, double eta,
    double* __restrict__ g) {
  using T2 = typename CT<R>::T2;
  extern __shared__ unsigned char smraw[];
  T2* rs = reinterpret_cast<T2*>(smraw);          // [nG][PCH]
  T2* us = rs + (size_t)nG * PCH;                  // [nG][WT]
  T2* vs = us + (size_t)nG * WT;                   // [nG][WT]
  constexpr int NWT = WT / OG;                     // frequencies per thread
  const int lane = threadIdx.x & 31, og = threadIdx.x >> 5;
  const int w0 = blockIdx.y * WT;
  for (int e = threadIdx.x; e < nG * WT; e += blockDim.x) {
    const int G = e / WT, j = e % WT;
    const int w = w0 + j;
    double2 a = make_double2(0, 0), c = make_double2(0, 0);
    if (w < nwi) {
      a = u[(size_t)w * nG + G];
      c = v[(size_t)w * nG + G];
    }
    us[e] = T2{(R)a.x, (R)a.y};
    vs[e] = T2{(R)c.x, (R)c.y};
  }
  // frequencies of this thread, as (hi, lo) so that w + Delta keeps its accuracy in FP32
  R wh[NWT], wl[NWT];
  for (int i = 0; i < NWT; ++i) {
    const int w = w0 + og * NWT + i;
    const double f = w < nwi ? freqs[w] : 0.0;
    wh[i] = (R)f;
    wl[i] = (R)(f - (double)wh[i]);
  }
  double accT[NWT][2], accE[NWT][2];
  R parT[NWT][2], parE[NWT][2];
  for (int i = 0; i < NWT; ++i) {
    accT[i][0] = accT[i][1] = accE[i][0] = accE[i][1] = 0.0;
    parT[i][0] = parT[i][1] = parE[i][0] = parE[i][1] = (R)0;
  }
  const long long pb = (long long)blockIdx.x * per_split;
  const long long pe = min(np, pb + per_split);
  int nchunk = 0;
  const R e = (R)eta;
  for (long long p0 = pb; p0 < pe; p0 += PCH) {
    __syncthreads();
    for (int e2 = threadIdx.x; e2 < nG * PCH; e2 += blockDim.x) {
      const int G = e2 / PCH, l = e2 % PCH;
      const long long p = p0 + l;
      T2 val = T2{(R)0, (R)0};
      if (p < pe) {
        if (gpad)
          val = rho[((size_t)((p >> 5) * gpad + G) << 5) + (size_t)(p & 31)];
        else
          val = rho[(size_t)G * ld + (size_t)p];
      }
      rs[e2] = val;
    }
    __syncthreads();
    const long long p = p0 + lane;
    if (p >= pe) continue;
    R ar[NWT], ai[NWT], br[NWT], bi[NWT];
    for (int i = 0; i < NWT; ++i) ar[i] = ai[i] = br[i] = bi[i] = (R)0;
    for (int G = 0; G < nG; ++G) {
      const T2 r = rs[G * PCH + lane];
#pragma unroll
      for (int i = 0; i < NWT; ++i) {
        const T2 uu = us[G * WT + og * NWT + i];
        const T2 vv = vs[G * WT + og * NWT + i];
        // a += u rho ; b += conj(rho) v
        ar[i] += uu.x * r.x - uu.y * r.y;
        ai[i] += uu.x * r.y + uu.y * r.x;
        br[i] += r.x * vv.x + r.y * vv.y;
        bi[i] += r.x * vv.y - r.y * vv.x;
      }
    }
    const double dlt = delta[p];
    const R dh = (R)dlt, dl = (R)(dlt - (double)dh);
    const R dfp = (R)df[p], ddfp = (R)ddf[p];
#pragma unroll
    for (int i = 0; i < NWT; ++i) {
      const R tr = ar[i] * br[i] - ai[i] * bi[i], ti = ar[i] * bi[i] + ai[i] * br[i];
      const R x = (wh[i] + dh) + (wl[i] + dl);        // Re den
      const R d2 = x * x + e * e;                      // |den|^2
      const R inv = (R)1 / d2;
      // 1/den = (x - i e)/d2 ;  ddf/den
      const R cr = ddfp * x * inv, ci = -ddfp * e * inv;
      parT[i][0] += tr * cr - ti * ci;
      parT[i][1] += tr * ci + ti * cr;
      // -i df/den^2 = -i df (x - i e)^2 / d2^2 = df (-2 x e - i (x^2 - e^2)) / d2^2
      const R inv2 = inv * inv;
      const R qr = -(R)2 * dfp * x * e * inv2, qi = -dfp * (x * x - e * e) * inv2;
      parE[i][0] += tr * qr - ti * qi;
      parE[i][1] += tr * qi + ti * qr;
    }
    if (++nchunk == 64) {   // fold the FP32 partial sums into FP64 every 64 chunks
      nchunk = 0;
      for (int i = 0; i < NWT; ++i)
        for (int c = 0; c < 2; ++c) {
          accT[i][c] += (double)parT[i][c];
          accE[i][c] += (double)parE[i][c];
          parT[i][c] = parE[i][c] = (R)0;
        }
    }
  }
  for (int i = 0; i < NWT; ++i)
    for (int c = 0; c < 2; ++c) {
      double t = accT[i][c] + (double)parT[i][c];
      double s = accE[i][c] + (double)parE[i][c];
      for (int off = 16; off > 0; off >>= 1) {
        t += __shfl_down_sync(0xffffffffu, t, off);
        s += __shfl_down_sync(0xffffffffu, s, off);
      }
      const int w = w0 + og * NWT + i;
      if (lane == 0 && w < nwi) {
        atomicAdd(&g[(size_t)w * 4 + c], t);
        atomicAdd(&g[(size_t)w * 4 + 2 + c], s);
      }
    }
}

template <typename R, int WT>
lrt_status launch_project(const lrt_ctx* c, const QData& q, const double2* du, const double2* dv,
                          const double* ddelta, const double* ddf0, const double* dddf, double* dg,
                          cudaStream_t s) {
  using T2 = typename CT<R>::T2;
  const int nG = q.nG;
  const size_t smem = (size_t)nG * (PCH + 2 * WT) * sizeof(T2);
  if (smem > kProjSmem) {
    set_error("adjoint projections: N_G too large");
    return LRT_EUNSUPPORTED;
  }
  auto kern = adjoint_project_kernel<R, WT>;
  LRT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int ny = (c->nwi + WT - 1) / WT;
  long long nx = std::max<long long>(1, (8LL * nsm + ny - 1) / ny);
  long long per = (c->np + nx - 1) / nx;
  per = (per + PCH - 1) / PCH * PCH;
  nx = (c->np + per - 1) / per;
  dim3 grid((unsigned)nx, (unsigned)ny);
  kern<<<grid, 256, smem, s>>>((const T2*)c->dw.rho, c->rho_ld, c->rho_gpad, nG, du, dv, c->dw.freqs,
                               c->nwi, ddelta, ddf0, dddf, c->np, per, c->eta, dg);
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  return LRT_OK;
}

}  // namespace

// d chi_00(q, w)/d theta for one q at all internal frequencies: out[nwi][5] complex as
// (re, im) pairs, and q.ds0, the tangents of d chi_00/d eta at w = 0 (zerofreq.cu).  Needs
// chi0 and chi of the q and the pair densities of the q in dw.rho.
lrt_status launch_adjoint_q(const lrt_ctx* c, QData& q, int iq, std::vector<double>& out,
                            cudaStream_t s) {
  (void)iq;
  const int N = q.nG, nwi = c->nwi;
  const size_t nh = (size_t)c->nk * c->nb;
  // host: d mu/dT from the k-mesh states (band weights), unless the occupations are fixed
  const bool fixed = std::isnan(q.mu);
  double mup = 0.0;
  if (!fixed) {
    std::vector<double> e(nh), f(nh);
    LRT_CUDA(cudaMemcpy(e.data(), q.eps, nh * sizeof(double), cudaMemcpyDeviceToHost));
    LRT_CUDA(cudaMemcpy(f.data(), q.occ, nh * sizeof(double), cudaMemcpyDeviceToHost));
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < nh; ++i) {
      const double g = q.wgt_h[i] * f[i] * (1.0 - f[i]);
      num += g * (e[i] - q.mu);
      den += g;
    }
    mup = den > 0.0 ? -num / (c->T * den) : 0.0;
  }
  // kernel tangents dK/d(A, B, C)
  std::vector<double> dK(3 * (size_t)N, 0.0);
  if (c->kernel.kind == LRT_KERNEL_FXC_MODEL) {
    for (int g = 0; g < N; ++g) {
      const double qg2 = q.qg2[g];
      const double ex = std::exp(-c->kernel.C * qg2);
      dK[g] = c->fxc * (1.0 + c->kernel.B * qg2) * ex;
      dK[N + g] = c->kernel.A * c->fxc * qg2 * ex;
      dK[2 * N + g] = -c->kernel.A * c->fxc * (1.0 + c->kernel.B * qg2) * qg2 * ex;
    }
  }
  double *d_dK = nullptr, *d_dl = nullptr, *d_df = nullptr, *d_ddf = nullptr, *d_g = nullptr;
  double2 *d_u = nullptr, *d_v = nullptr, *d_k3 = nullptr, *d_ws = nullptr;
  auto freeall = [&]() {
    cudaFree(d_dK);
    cudaFree(d_dl);
    cudaFree(d_df);
    cudaFree(d_ddf);
    cudaFree(d_g);
    cudaFree(d_u);
    cudaFree(d_v);
    cudaFree(d_k3);
    cudaFree(d_ws);
  };
  auto fail = [&](cudaError_t e) {
    freeall();
    set_error(std::string("adjoint: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LRT_ENOMEM : LRT_ECUDA;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&d_dK, dK.size() * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&d_dl, c->np * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&d_df, c->np * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&d_ddf, c->np * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&d_g, (size_t)nwi * 4 * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&d_u, (size_t)nwi * N * sizeof(double2))) != cudaSuccess ||
      (e = cudaMalloc(&d_v, (size_t)nwi * N * sizeof(double2))) != cudaSuccess ||
      (e = cudaMalloc(&d_k3, (size_t)nwi * 3 * sizeof(double2))) != cudaSuccess)
    return fail(e);
  if ((e = cudaMemcpyAsync(d_dK, dK.data(), dK.size() * sizeof(double), cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemsetAsync(d_g, 0, (size_t)nwi * 4 * sizeof(double), s)) != cudaSuccess)
    return fail(e);
  const size_t mat = (size_t)N * (N + 1) * sizeof(double2);
  const size_t smem = mat + 2 * (size_t)N * sizeof(double2);
  if (smem > 227 * 1024) {
    // M^T in global memory: one slice per block, two blocks per SM
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return fail(e);
    const int grid = std::max(1, std::min(nwi, 2 * nsm));
    if ((e = cudaMalloc(&d_ws, (size_t)grid * mat)) != cudaSuccess) return fail(e);
    dyson_adjoint_kernel<true><<<grid, 256, 2 * (size_t)N * sizeof(double2), s>>>(
        q.chi0, q.Kdev, d_dK, q.chi, N, nwi, d_u, d_v, d_k3, c->dw.status, d_ws);
  } else {
    if ((e = cudaFuncSetAttribute(dyson_adjoint_kernel<false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return fail(e);
    dyson_adjoint_kernel<false><<<nwi, 256, smem, s>>>(q.chi0, q.Kdev, d_dK, q.chi, N, nwi, d_u,
                                                       d_v, d_k3, c->dw.status, nullptr);
  }
  count_launch(c);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  adjoint_pair_weights<<<1216, 256, 0, s>>>(q.eps, q.occ, q.wgt, c->nk, c->nb, q.mu, c->T, mup,
                                            fixed ? 1 : 0, d_dl, d_df, d_ddf);
  count_launch(c);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  // frequency tiles of 16 (FP64) or 32 (split) while the tile fits the shared memory, half
  // that above (N_G up to 266 for FP64, 400 for the split path)
  const bool wide64 = (size_t)N * (PCH + 2 * 16) * sizeof(double2) <= kProjSmem;
  const bool wide32 = (size_t)N * (PCH + 2 * 32) * sizeof(float2) <= kProjSmem;
  lrt_status st;
  if (c->precision == LRT_PREC_FP64)
    st = wide64 ? launch_project<double, 16>(c, q, d_u, d_v, d_dl, d_df, d_ddf, d_g, s)
                : launch_project<double, 8>(c, q, d_u, d_v, d_dl, d_df, d_ddf, d_g, s);
  else
    st = wide32 ? launch_project<float, 32>(c, q, d_u, d_v, d_dl, d_df, d_ddf, d_g, s)
                : launch_project<float, 16>(c, q, d_u, d_v, d_dl, d_df, d_ddf, d_g, s);
  if (st != LRT_OK) {
    freeall();
    return st;
  }
  // the w -> 0 limit S(0) = (T/(pi n)) Re d chi_00/d eta: its tangents are second derivatives
  q.ds0.assign(10, 0.0);
  st = launch_s0_tangents(c, q, d_u + (size_t)c->hcol * N, d_v + (size_t)c->hcol * N, d_dK, d_dl,
                          d_df, d_ddf, q.ds0.data(), s);
  if (st != LRT_OK) {
    freeall();
    return st;
  }
  std::vector<double> g((size_t)nwi * 4);
  std::vector<double2> k3((size_t)nwi * 3);
  if ((e = cudaMemcpyAsync(g.data(), d_g, g.size() * sizeof(double), cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(k3.data(), d_k3, k3.size() * sizeof(double2), cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return fail(e);
  freeall();
  const double rs = (c->precision == LRT_PREC_FP64) ? 1.0 : (double)split_rho_scale(c->precision);
  const double pref = 2.0 / (c->nk * c->volume) / (rs * rs);
  out.assign((size_t)nwi * 10, 0.0);
  for (int w = 0; w < nwi; ++w) {
    double* o = &out[(size_t)w * 10];
    o[0] = pref * g[(size_t)w * 4 + 0];
    o[1] = pref * g[(size_t)w * 4 + 1];
    o[2] = pref * g[(size_t)w * 4 + 2];
    o[3] = pref * g[(size_t)w * 4 + 3];
    for (int j = 0; j < 3; ++j) {
      o[4 + 2 * j] = k3[(size_t)w * 3 + j].x;
      o[5 + 2 * j] = k3[(size_t)w * 3 + j].y;
    }
  }
  return LRT_OK;
}

}  // namespace lrt
