// S(q,w) by the fluctuation-dissipation theorem (Eq. 8) and F(q,tau) by the two-sided
// Laplace transform (Eq. 1), FP64, one warp per output with a shuffle reduction.
//   S(q,w) = -Im chi_00(q,w) / (pi n (1 - e^{-w/T})), the denominator as -expm1(-w/T);
//   S(q,0) = (T/(pi n)) Re s0, s0 = d chi_00/d eta at w = 0 (the w -> 0 limit, zerofreq.cu).
//   FOLD:   F(tau) = sum_i wt_i S_i [e^{-tau w_i} + e^{-(beta - tau) w_i}] over the w >= 0
//           samples plus w = 0 (detailed balance S(-w) = e^{-beta w} S(w)), trapezoid wt;
//   DIRECT: F(tau) = sum_j wt_j S_j e^{-tau w_j} over the caller's grid.
//   metrics: F(beta/2), int_0^beta F, F~(beta/2) = F(beta/2) - F(0) (Eq. 2),
//            int_0^beta F~ = int F - beta F(0), chi_static = -n int_0^beta F (Sec. 2), with
//            int_0^beta [e^{-tau w} + e^{-(beta-tau) w}] dtau = 2 (1 - e^{-beta w}) / w.
#include "lrt_internal.h"

namespace lrt {
namespace {

// rows r = (q, eta) of S: chi00 [rows][nwi], s0 [rows], S [rows][nw]
__global__ void dsf_kernel(const double2* __restrict__ chi00, const double2* __restrict__ s0,
                           const double* __restrict__ omega, int nq, int nw, int nwi, double T,
                           double n, double* __restrict__ S) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nq * nw) return;
  int iq = t / nw, j = t % nw;
  double w = omega[j];
  const double2* c = chi00 + (size_t)iq * nwi;
  double v;
  if (w == 0.0)
    v = T * s0[iq].x / (M_PI * n);
  else
    v = -c[j].y / (M_PI * n * (-expm1(-w / T)));
  S[t] = v;
}

// Positive branch: sample i of q (i = 0..npos-1) -> (w_i, S_i).
struct Branch {
  int jp;        // first caller index with w >= 0
  int zero;      // 1 when w = 0 is on the caller's grid
  int npos;      // samples in the branch
};

__device__ inline void branch_point(const Branch& b, const double* omega, const double* Sq,
                                    double S0, int i, double* x, double* y) {
  if (b.zero) {
    *x = omega[b.jp + i];
    *y = Sq[b.jp + i];
  } else if (i == 0) {
    *x = 0.0;
    *y = S0;
  } else {
    *x = omega[b.jp + i - 1];
    *y = Sq[b.jp + i - 1];
  }
}

__device__ inline double branch_weight(const Branch& b, const double* omega, int i) {
  double xm, xp, x, dummy;
  branch_point(b, omega, omega, 0.0, i, &x, &dummy);
  double w = 0.0;
  if (i > 0) {
    branch_point(b, omega, omega, 0.0, i - 1, &xm, &dummy);
    w += 0.5 * (x - xm);
  }
  if (i < b.npos - 1) {
    branch_point(b, omega, omega, 0.0, i + 1, &xp, &dummy);
    w += 0.5 * (xp - x);
  }
  return w;
}

__device__ inline double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// one warp per (q, tau)
__global__ void itcf_fold_kernel(const double* __restrict__ S, const double2* __restrict__ s0,
                                 const double* __restrict__ omega, const double* __restrict__ tau,
                                 Branch b, int nq, int nw, int ntau, double T, double n,
                                 double* __restrict__ F) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= nq * ntau) return;
  int iq = warp / ntau, it = warp % ntau;
  const double beta = 1.0 / T;
  const double* Sq = S + (size_t)iq * nw;
  const double S0 = T * s0[iq].x / (M_PI * n);
  double ta = tau[it];
  double acc = 0.0;
  for (int i = lane; i < b.npos; i += 32) {
    double x, y;
    branch_point(b, omega, Sq, S0, i, &x, &y);
    acc += branch_weight(b, omega, i) * y * (exp(-ta * x) + exp(-(beta - ta) * x));
  }
  acc = warp_sum(acc);
  if (lane == 0) F[(size_t)iq * ntau + it] = acc;
}

__global__ void itcf_direct_kernel(const double* __restrict__ S, const double* __restrict__ omega,
                                   const double* __restrict__ tau, int nq, int nw, int ntau,
                                   double* __restrict__ F) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= nq * ntau) return;
  int iq = warp / ntau, it = warp % ntau;
  const double* Sq = S + (size_t)iq * nw;
  double ta = tau[it];
  double acc = 0.0;
  for (int j = lane; j < nw; j += 32) {
    double wt = 0.0;
    if (j > 0) wt += 0.5 * (omega[j] - omega[j - 1]);
    if (j < nw - 1) wt += 0.5 * (omega[j + 1] - omega[j]);
    acc += wt * Sq[j] * exp(-ta * omega[j]);
  }
  acc = warp_sum(acc);
  if (lane == 0) F[(size_t)iq * ntau + it] = acc;
}

// one warp per q
__global__ void itcf_metrics_kernel(const double* __restrict__ S, const double2* __restrict__ s0,
                                    const double* __restrict__ omega, Branch b, int nq, int nw,
                                    double T, double n, double* __restrict__ metrics) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= nq) return;
  const int iq = warp;
  const double beta = 1.0 / T;
  const double* Sq = S + (size_t)iq * nw;
  const double S0 = T * s0[iq].x / (M_PI * n);
  double fh = 0.0, f0 = 0.0, fi = 0.0;
  for (int i = lane; i < b.npos; i += 32) {
    double x, y;
    branch_point(b, omega, Sq, S0, i, &x, &y);
    double wy = branch_weight(b, omega, i) * y;
    fh += wy * 2.0 * exp(-0.5 * beta * x);
    f0 += wy * (1.0 + exp(-beta * x));
    fi += wy * (x > 0.0 ? -2.0 * expm1(-beta * x) / x : 2.0 * beta);
  }
  fh = warp_sum(fh);
  f0 = warp_sum(f0);
  fi = warp_sum(fi);
  if (lane == 0) {
    double* m = metrics + (size_t)iq * 5;
    m[0] = fh;
    m[1] = fi;
    m[2] = fh - f0;
    m[3] = fi - beta * f0;
    m[4] = -n * fi;
  }
}

__global__ void gather_chi00(const double2* __restrict__ chi, int nG, int nwi,
                             double2* __restrict__ out) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < nwi) out[w] = chi[(size_t)w * nG];
}

Branch make_branch(const lrt_ctx* c) {
  Branch b;
  b.jp = c->nw;
  for (int j = 0; j < c->nw; ++j)
    if (c->omega[j] >= 0.0) {
      b.jp = j;
      break;
    }
  b.zero = (b.jp < c->nw && c->omega[b.jp] == 0.0) ? 1 : 0;
  b.npos = (c->nw - b.jp) + (b.zero ? 0 : 1);
  return b;
}

// Reference eta of each q (Sec. 2): the largest eta_j such that for every i <= j both
// F~(beta/2) and int_0^beta F~ (metrics 2 and 3) lie within tol |m(eta_0)| of their value at
// the smallest eta.  One thread per q; metrics [nq][neta][5].
__global__ void eta_pick_kernel(const double* __restrict__ metrics, int nq, int neta, double tol,
                                int* __restrict__ ref) {
  int iq = blockIdx.x * blockDim.x + threadIdx.x;
  if (iq >= nq) return;
  const double* m = metrics + (size_t)iq * neta * 5;
  int r = 0;
  for (int j = 1; j < neta; ++j) {
    bool ok = true;
    for (int k = 2; k <= 3; ++k)
      if (fabs(m[j * 5 + k] - m[k]) > tol * fabs(m[k])) ok = false;
    if (!ok) break;   // the earlier etas already passed
    r = j;
  }
  ref[iq] = r;
}

}  // namespace

lrt_status launch_eta_pick(const lrt_ctx* c, const double* metrics_dev, int nq, int neta, double tol,
                           int* ref_dev, cudaStream_t s) {
  eta_pick_kernel<<<(nq + 127) / 128, 128, 0, s>>>(metrics_dev, nq, neta, tol, ref_dev);
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  return LRT_OK;
}

// S rows are (q, eta) pairs, q-major: row q neta + j holds eta j of q (one row per q for a
// single eta); F and the metrics follow the same rows.
lrt_status launch_dsf(const lrt_ctx* c, double* S_dev, cudaStream_t s) {
  const int nc = ncol(c);
  for (int iq = 0; iq < c->nq; ++iq) {
    gather_chi00<<<(nc + 255) / 256, 256, 0, s>>>(c->qd[iq].chi, c->qd[iq].nG, nc,
                                                  (double2*)c->dw.chi00 + (size_t)iq * nc);
    LRT_CUDA(cudaGetLastError());
  }
  const int rows = nrow(c);
  int total = rows * c->nw;
  dsf_kernel<<<(total + 255) / 256, 256, 0, s>>>((const double2*)c->dw.chi00, c->dw.s0, c->dw.omega,
                                                 rows, c->nw, c->nwi, c->T, c->density, S_dev);
  count_launch(c, c->nq + 1);
  LRT_CUDA(cudaGetLastError());
  return LRT_OK;
}

lrt_status launch_itcf(const lrt_ctx* c, const double* S_dev, int ntau, const double* tau_dev,
                       int mode, double* F_dev, double* metrics_dev, cudaStream_t s) {
  return launch_itcf_rows(c, S_dev, c->dw.s0, nrow(c), ntau, tau_dev, mode, F_dev, metrics_dev, s);
}

lrt_status launch_itcf_rows(const lrt_ctx* c, const double* S_dev, const double2* s0_dev, int rows,
                            int ntau, const double* tau_dev, int mode, double* F_dev,
                            double* metrics_dev, cudaStream_t s) {
  Branch b = make_branch(c);
  if (mode == LRT_ITCF_FOLD && b.npos < 2) {
    set_error("FOLD needs at least one sample with w > 0");
    return LRT_EINVAL;
  }
  int warps = rows * ntau;
  int blocks = (warps * 32 + 255) / 256;
  if (mode == LRT_ITCF_FOLD)
    itcf_fold_kernel<<<blocks, 256, 0, s>>>(S_dev, s0_dev, c->dw.omega, tau_dev, b, rows, c->nw,
                                            ntau, c->T, c->density, F_dev);
  else
    itcf_direct_kernel<<<blocks, 256, 0, s>>>(S_dev, c->dw.omega, tau_dev, rows, c->nw, ntau, F_dev);
  count_launch(c, metrics_dev ? 2 : 1);
  LRT_CUDA(cudaGetLastError());
  if (metrics_dev) {
    int mb = (rows * 32 + 255) / 256;
    itcf_metrics_kernel<<<mb, 256, 0, s>>>(S_dev, s0_dev, c->dw.omega, b, rows, c->nw, c->T,
                                           c->density, metrics_dev);
    LRT_CUDA(cudaGetLastError());
  }
  return LRT_OK;
}

}  // namespace lrt
