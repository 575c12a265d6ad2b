// Dyson equation chi = (1 - chi0 K)^{-1} chi0 with K diagonal, FP64: for each frequency one
// block loads M = 1 - chi0 K (M_GG' = delta_GG' - chi0_GG' K_G') and solves M x = chi0_{:,0} by
// Gaussian elimination with partial pivoting (pivot = largest modulus, first on ties) and back
// substitution; x = chi_{G,0}.  M sits in shared memory while it fits (N_G <= 118); above that
// each block keeps it in its own slice of a global workspace (L2-resident for the sizes of
// interest) and loops over frequencies.  Both forms run the same operations in the same order.
// A zero pivot sets bit 1 of the device status word and leaves NaN in x.
#include <algorithm>

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

// Block loop over frequencies w = blockIdx.x, blockIdx.x + gridDim.x, ...  GM: M in ws
// (N x (N+1) per block), shared memory rhs[N], fac[N]; otherwise shared memory N x (N+1)
// matrix, then rhs[N], fac[N].
template <bool GM>
__global__ void __launch_bounds__(256) dyson_kernel(const double2* __restrict__ chi0,
                                                    const double* __restrict__ K, int N, int nw,
                                                    double2* __restrict__ chi,
                                                    int* __restrict__ status, double2* ws) {
  extern __shared__ double2 sm[];
  const int ld = N + 1;
  double2* M = GM ? ws + (size_t)blockIdx.x * N * ld : sm;
  double2* b = GM ? sm : sm + (size_t)N * ld;
  double2* fac = b + N;
  __shared__ int piv_s;
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) bad = 0;
  for (int w = blockIdx.x; w < nw; w += gridDim.x) {
    const double2* X = chi0 + (size_t)w * N * N;
    __syncthreads();   // the previous frequency's back substitution is done with M and b
    for (int e = tid; e < N * N; e += nt) {
      int r = e / N, j = e % N;
      double2 v = X[e];
      double2 m = make_double2(-v.x * K[j], -v.y * K[j]);
      if (r == j) m.x += 1.0;
      M[r * ld + j] = m;
      if (j == 0) b[r] = v;
    }
    __syncthreads();
    for (int c = 0; c < N; ++c) {
      if (tid < 32) {
        double best = -1.0;
        int bi = c;
        for (int r = c + tid; r < N; r += 32) {
          double2 v = M[r * ld + c];
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
          double2 t = M[c * ld + j];
          M[c * ld + j] = M[p * ld + j];
          M[p * ld + j] = t;
        }
        if (tid == 0) {
          double2 t = b[c];
          b[c] = b[p];
          b[p] = t;
        }
      }
      __syncthreads();
      const double2 d = M[c * ld + c];
      for (int r = c + 1 + tid; r < N; r += nt) fac[r] = cdiv(M[r * ld + c], d);
      __syncthreads();
      const int rows = N - c - 1;
      const int cols = N - c;  // columns c+1..N-1 plus the rhs
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
          double2 t = cmul(f, M[c * ld + j]);
          M[r * ld + j].x -= t.x;
          M[r * ld + j].y -= t.y;
        }
      }
      __syncthreads();
    }
    // back substitution, column oriented
    for (int c = N - 1; c >= 0; --c) {
      if (tid == 0) b[c] = cdiv(b[c], M[c * ld + c]);
      __syncthreads();
      const double2 xc = b[c];
      for (int r = tid; r < c; r += nt) {
        double2 t = cmul(M[r * ld + c], xc);
        b[r].x -= t.x;
        b[r].y -= t.y;
      }
      __syncthreads();
    }
    for (int r = tid; r < N; r += nt) chi[(size_t)w * N + r] = b[r];
  }
  if (tid == 0 && bad) atomicOr(status, 1);
}

}  // namespace

lrt_status launch_dyson(const lrt_ctx* c, QData& q, int iq, cudaStream_t s) {
  (void)iq;
  const int N = q.nG, nw = ncol(c);   // every internal frequency of every eta
  const size_t mat = (size_t)N * (N + 1) * sizeof(double2);
  const size_t smem = mat + 2 * (size_t)N * sizeof(double2);
  int dev = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  if (smem > 227 * 1024) {
    // global-memory form: one matrix slice per block, two blocks per SM; the workspace is
    // allocated on the first call that needs it (before any graph capture: the capture
    // follows an ordinary pass)
    int nsm = 0;
    LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::max(1, std::min(nw, 2 * nsm));
    lrt_ctx* cc = const_cast<lrt_ctx*>(c);
    if (cc->dw.dyson_bytes < (size_t)grid * mat) {
      cudaFree(cc->dw.dyson_ws);
      cc->dw.dyson_ws = nullptr;
      cc->dw.dyson_bytes = 0;
      LRT_CUDA(cudaMalloc(&cc->dw.dyson_ws, (size_t)grid * mat));
      cc->dw.dyson_bytes = (size_t)grid * mat;
    }
    dyson_kernel<true><<<grid, 256, 2 * (size_t)N * sizeof(double2), s>>>(
        q.chi0, q.Kdev, N, nw, q.chi, c->dw.status, (double2*)cc->dw.dyson_ws);
    count_launch(c);
    LRT_CUDA(cudaGetLastError());
    return LRT_OK;
  }
  // raised only when a call needs more than any earlier one on this device, so repeated
  // calls (and a graph capture after a first pass) make no attribute call
  static size_t attr_set[64] = {0};
  if (dev < 0 || dev >= 64 || attr_set[dev] < smem) {
    LRT_CUDA(cudaFuncSetAttribute(dyson_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    if (dev >= 0 && dev < 64) attr_set[dev] = smem;
  }
  dyson_kernel<false><<<nw, 256, smem, s>>>(q.chi0, q.Kdev, N, nw, q.chi, c->dw.status, nullptr);
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  return LRT_OK;
}

}  // namespace lrt
