// Dielectric properties from a (filtered) dynamic structure factor: Sec. 3 (after the
// workflow figure) and App. A.2, Eqs. 10 and 11.
//   Im chi(q,w) = -pi n (1 - e^{-w/T}) S(q,w)                    (Eq. 8 solved for Im chi)
//   Re chi(q,w) = (2/pi) P int_0^inf w' Im chi(q,w') / (w'^2 - w^2) dw'   (Kramers-Kronig; Im chi
//                 is odd in w)
//   1/eps = 1 + (4 pi/q^2) chi  (Eq. 10),   sigma = (i w/(4 pi)) (1 - eps)  (Eq. 11)
// on the uniformly spaced samples w_j >= 0 of the caller's grid (spacing h).  The principal
// value is taken by Maclaurin's formula (Ohta and Ishida, Appl. Spectrosc. 42, 952 (1988)):
//   Re chi(w_i) = (2/pi) 2h sum_{j: i - j odd} w_j Im chi(w_j) / (w_j^2 - w_i^2),
// which never evaluates the singular node; the integral below the first sample and above the
// last one is left out (truncation).  One warp per output sample, FP64.
#include <cmath>
#include <vector>

#include "lrt_internal.h"

namespace lrt {
namespace {

// rows of S [rows][nw]; samples jp .. jp + N - 1 are w >= 0; vq[row] = 4 pi/|q|^2;
// out [rows][N][8] = Re chi, Im chi, Re 1/eps, Im 1/eps, Re eps, Im eps, Re sigma, Im sigma
__global__ void __launch_bounds__(256) dielectric_kernel(const double* __restrict__ S,
                                                          const double* __restrict__ omega,
                                                          const double* __restrict__ vq, int rows,
                                                          int nw, int jp, int N, double h, double T,
                                                          double n, double* __restrict__ out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= rows * N) return;
  const int r = warp / N, i = warp % N;
  const double* Sr = S + (size_t)r * nw + jp;
  const double* w = omega + jp;
  const double wi = w[i];
  double acc = 0.0;
  for (int j = (i + 1) % 2 + 2 * lane; j < N; j += 64) {   // nodes of the other parity
    const double wj = w[j];
    const double im = -M_PI * n * (-expm1(-wj / T)) * Sr[j];
    acc += wj * im / (wj * wj - wi * wi);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane != 0) return;
  const double re = (2.0 / M_PI) * 2.0 * h * acc;
  const double im = -M_PI * n * (-expm1(-wi / T)) * Sr[i];
  // 1/eps = 1 + v chi;  eps = 1/(1/eps);  sigma = (i w/(4 pi)) (1 - eps)
  const double v = vq[r];
  const double ar = 1.0 + v * re, ai = v * im;
  const double d = ar * ar + ai * ai;
  const double er = ar / d, ei = -ai / d;
  const double sr = -wi / (4.0 * M_PI) * (-ei), si = wi / (4.0 * M_PI) * (1.0 - er);
  double* o = out + ((size_t)r * N + i) * 8;
  o[0] = re;
  o[1] = im;
  o[2] = ar;
  o[3] = ai;
  o[4] = er;
  o[5] = ei;
  o[6] = sr;
  o[7] = si;
}

}  // namespace

lrt_status run_dielectric(const lrt_ctx* c, const double* S, int rows, const double* vq, double* out) {
  int jp = c->nw;
  for (int j = 0; j < c->nw; ++j)
    if (c->omega[j] >= 0.0) {
      jp = j;
      break;
    }
  const int N = c->nw - jp;
  if (N < 3) {
    set_error("the Kramers-Kronig transform needs at least 3 samples with w >= 0");
    return LRT_EINVAL;
  }
  const double h = c->omega[jp + 1] - c->omega[jp];
  for (int j = jp + 1; j < c->nw; ++j)
    if (std::fabs((c->omega[j] - c->omega[j - 1]) - h) > 1e-9 * h) {
      set_error("the Kramers-Kronig transform needs uniformly spaced samples with w >= 0");
      return LRT_EINVAL;
    }
  LRT_CUDA(cudaSetDevice(c->device));
  double *dS = nullptr, *dv = nullptr, *dout = nullptr;
  auto done = [&](lrt_status st) {
    cudaFree(dS);
    cudaFree(dv);
    cudaFree(dout);
    return st;
  };
  const size_t nout = (size_t)rows * N * 8;
  if (cudaMalloc(&dS, (size_t)rows * c->nw * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dv, rows * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dout, nout * sizeof(double)) != cudaSuccess) {
    set_error("device allocation");
    return done(LRT_ENOMEM);
  }
  if (cudaMemcpy(dS, S, (size_t)rows * c->nw * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dv, vq, rows * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return done(LRT_ECUDA);
  const long long warps = (long long)rows * N;
  dielectric_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256>>>(dS, c->dw.omega, dv, rows, c->nw, jp,
                                                                   N, h, c->T, c->density, dout);
  count_launch(c);
  if (cudaGetLastError() != cudaSuccess) return done(LRT_ECUDA);
  if (cudaMemcpy(out, dout, nout * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return done(LRT_ECUDA);
  return done(LRT_OK);
}

}  // namespace lrt

using namespace lrt;

extern "C" lrt_status lrtddft_dielectric(lrt_ctx* c, const double* S, double* out) {
  if (!c || !S || !out) {
    set_error("NULL argument");
    return LRT_EINVAL;
  }
  if (c->host_only) {
    set_error("host-only context");
    return LRT_ESTATE;
  }
  const int rows = nrow(c);
  std::vector<double> vq(rows);
  for (int r = 0; r < rows; ++r) {
    const double* q = &c->q[3 * (size_t)(r / c->neta)];
    vq[r] = 4.0 * M_PI / (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
  }
  return run_dielectric(c, S, rows, vq.data(), out);
}
