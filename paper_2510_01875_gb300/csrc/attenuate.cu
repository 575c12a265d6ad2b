// Constraints-based attenuation of narrow-band fluctuations (Sec. 3), FP64, on the
// uniformly spaced samples with w >= 0 of each q's DSF.
//
//  prep (block per q):    dS/dw by central differences over the featureless range, its
//                         Hann-windowed periodogram (direct DFT), the n_targets strongest local
//                         maxima above the lowest low_exclude of the frequencies, the +-2 bin
//                         neighbourhoods of the targets and their raw power, and the raw sum of
//                         squared second differences.
//  candidates (block per (candidate, q)): the Savitzky-Golay smoother of degree d over m
//                         points from the normal equations of the local polynomial fit
//                         (Gram matrix of t = offset/h, inverted by Gauss-Jordan): interior
//                         weights c_j = [G^-1 v(t_j)]_0, edge rows evaluate the first / last
//                         window's polynomial; then RSS, trace of the smoother, AICc, the
//                         kept target power R_f of the filtered dS/dw, the second-difference
//                         ratio and the score AICc + lambda_f ln(max(R_f, r0)/r0) + lambda_c
//                         (curvature ratio); sign changes of the filtered dS/dw for ties.
//  select (block per q):  best window per degree (ties within 1e-9 relative -> fewer sign
//                         changes -> smaller window), F_n = Laplace transform of S - S_p on
//                         the tau grid (Eq. 5), Fbar_n and sigma_n (Eq. 7), acceptance against
//                         F(beta/2), S_p = mean (or best) of the accepted degrees.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "lrt_internal.h"

namespace lrt {
namespace {

constexpr int kMaxTargets = 4;
constexpr int kMaxBins = kMaxTargets * 5;
constexpr int kMaxDegree = 8;

struct AttQ {            // per-q result of the prep kernel
  int ntg;
  int tg[kMaxTargets];
  int nbins;
  int bins[kMaxBins];
  double raw_power;
  double curv_raw;
};

struct AttCfg {
  int N;                 // samples in the filtered run
  int jp;                // caller index of the first sample (w >= 0)
  int zero;              // 1 when w = 0 is sample 0; else the S(0) point precedes the run
  double dw;
  int i0, i1, L, K;      // derivative range and periodogram size
  int kmin;              // lowest periodogram bin searched for targets
  int ntargets;
  int ncand;
  double lf, lc, r0;
  int ndeg, dmin;
  int ntau;
  double accept_mean, accept_rms;
  int average;           // 1 mean of accepted degrees, 0 best score
  double T, n;
  int nw;
};

__device__ inline double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// periodogram bin k of x[0..L): |sum_j x_j e^{-2 pi i j k / L}|^2, phase reduced mod L
__device__ inline double dft_power(const double* x, int L, int k, double* red) {
  double re = 0.0, im = 0.0;
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    long long r = ((long long)j * k) % L;
    double s, c;
    sincospi(2.0 * (double)r / (double)L, &s, &c);
    re += x[j] * c;
    im -= x[j] * s;
  }
  re = block_sum(re, red);
  im = block_sum(im, red);
  return re * re + im * im;
}

__device__ inline double hann(int j, int L) {
  return 0.5 - 0.5 * cospi(2.0 * (double)j / (double)(L - 1));
}

// scratch per q: D[L] (windowed derivative), P[K+1]
__global__ void att_prep(const double* __restrict__ S, AttCfg cfg, double* __restrict__ work,
                         AttQ* __restrict__ out) {
  __shared__ double red[33];
  const int iq = blockIdx.x;
  const double* y = S + (size_t)iq * cfg.nw + cfg.jp;
  double* x = work + (size_t)iq * (cfg.L + cfg.K + 1);
  double* P = x + cfg.L;
  double mean = 0.0;
  for (int j = threadIdx.x; j < cfg.L; j += blockDim.x) {
    int jj = cfg.i0 + j;
    double d = (y[jj + 1] - y[jj - 1]) / (2.0 * cfg.dw);
    x[j] = d;
    mean += d;
  }
  mean = block_sum(mean, red) / cfg.L;
  for (int j = threadIdx.x; j < cfg.L; j += blockDim.x) x[j] = hann(j, cfg.L) * (x[j] - mean);
  __syncthreads();
  for (int k = 0; k <= cfg.K; ++k) {
    double p = dft_power(x, cfg.L, k, red);
    if (threadIdx.x == 0) P[k] = p;
  }
  double cr = 0.0;
  for (int j = 1 + threadIdx.x; j < cfg.N - 1; j += blockDim.x) {
    double d2 = y[j + 1] - 2.0 * y[j] + y[j - 1];
    cr += d2 * d2;
  }
  cr = block_sum(cr, red);
  __syncthreads();
  if (threadIdx.x == 0) {
    AttQ q;
    q.curv_raw = cr;
    // strongest local maxima, ties to the lower bin
    int best[kMaxTargets];
    int nb = 0;
    for (int k = cfg.kmin + 1; k < cfg.K; ++k) {
      if (!(P[k] > P[k - 1] && P[k] >= P[k + 1])) continue;
      int pos = nb;
      while (pos > 0 && (P[k] > P[best[pos - 1]])) --pos;
      if (pos >= cfg.ntargets) continue;
      int last = nb < cfg.ntargets ? nb : cfg.ntargets - 1;
      for (int i = last; i > pos; --i) best[i] = best[i - 1];
      best[pos] = k;
      if (nb < cfg.ntargets) ++nb;
    }
    // ascending order
    for (int i = 0; i < nb; ++i)
      for (int j = i + 1; j < nb; ++j)
        if (best[j] < best[i]) {
          int t = best[i];
          best[i] = best[j];
          best[j] = t;
        }
    q.ntg = nb;
    for (int i = 0; i < kMaxTargets; ++i) q.tg[i] = i < nb ? best[i] : -1;
    // union of +-2 neighbourhoods, ascending
    q.nbins = 0;
    for (int b = 0; b <= cfg.K; ++b) {
      bool in = false;
      for (int i = 0; i < nb; ++i)
        if (b >= best[i] - 2 && b <= best[i] + 2) in = true;
      if (in && q.nbins < kMaxBins) q.bins[q.nbins++] = b;
    }
    double rp = 0.0;
    for (int i = 0; i < q.nbins; ++i) rp += P[q.bins[i]];
    q.raw_power = rp;
    out[iq] = q;
  }
}

struct CandOut {
  double score;
  int sign_changes;
  int valid;
};

// Gauss-Jordan inverse of the (d+1)x(d+1) Gram matrix in place (symmetric positive definite)
__device__ void small_inverse(double* A, int n) {
  double inv[(kMaxDegree + 1) * (kMaxDegree + 1)];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) inv[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
    if (p != c)
      for (int j = 0; j < n; ++j) {
        double t = A[c * n + j];
        A[c * n + j] = A[p * n + j];
        A[p * n + j] = t;
        t = inv[c * n + j];
        inv[c * n + j] = inv[p * n + j];
        inv[p * n + j] = t;
      }
    double d = A[c * n + c];
    for (int j = 0; j < n; ++j) {
      A[c * n + j] /= d;
      inv[c * n + j] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[r * n + j] -= f * A[c * n + j];
        inv[r * n + j] -= f * inv[c * n + j];
      }
    }
  }
  for (int i = 0; i < n * n; ++i) A[i] = inv[i];
}

__device__ inline double poly_dot(const double* u, int n, double t) {
  double s = 0.0, tp = 1.0;
  for (int a = 0; a < n; ++a) {
    s += u[a] * tp;
    tp *= t;
  }
  return s;
}

// grid (ncand, nq); cands[c] = (d, m); yf scratch [nq][ncand][N]
__global__ void att_candidates(const double* __restrict__ S, AttCfg cfg, const int2* __restrict__ cands,
                               const AttQ* __restrict__ qinfo, double* __restrict__ yf_all,
                               double* __restrict__ dwork, CandOut* __restrict__ cout) {
  __shared__ double red[33];
  __shared__ double Ginv[(kMaxDegree + 1) * (kMaxDegree + 1)];
  __shared__ double hat_edge;
  const int ci = blockIdx.x, iq = blockIdx.y;
  const int d = cands[ci].x, m = cands[ci].y, h = m / 2, n = d + 1, N = cfg.N;
  const double* y = S + (size_t)iq * cfg.nw + cfg.jp;
  double* yf = yf_all + ((size_t)iq * cfg.ncand + ci) * N;
  double* x = dwork + ((size_t)iq * cfg.ncand + ci) * cfg.L;
  const AttQ Q = qinfo[iq];
  if (threadIdx.x == 0) {
    double G[(kMaxDegree + 1) * (kMaxDegree + 1)];
    double mom[2 * kMaxDegree + 1];
    for (int e = 0; e < 2 * n - 1; ++e) mom[e] = 0.0;
    for (int j = 0; j < m; ++j) {
      double t = (double)(j - h) / h, tp = 1.0;
      for (int e = 0; e < 2 * n - 1; ++e) {
        mom[e] += tp;
        tp *= t;
      }
    }
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) G[a * n + b] = mom[a + b];
    small_inverse(G, n);
    for (int i = 0; i < n * n; ++i) Ginv[i] = G[i];
  }
  __syncthreads();
  // interior: y_f[j] = sum_t c_t y[j + t], c_t = sum_a Ginv[0][a] t^a
  for (int j = h + threadIdx.x; j < N - h; j += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < m; ++r) s += poly_dot(Ginv, n, (double)(r - h) / h) * y[j - h + r];
    yf[j] = s;
  }
  // edges: row r of the first window (r < h) and row h+1+r of the last window
  double hsum = 0.0;
  for (int e = threadIdx.x; e < 2 * h; e += blockDim.x) {
    int row = e < h ? e : e + 1;                 // window row
    int base = e < h ? 0 : N - m;                // window start
    double tr = (double)(row - h) / h;
    double u[kMaxDegree + 1], v[kMaxDegree + 1];
    double tp = 1.0;
    for (int a = 0; a < n; ++a) {
      v[a] = tp;
      tp *= tr;
    }
    for (int a = 0; a < n; ++a) {
      double s = 0.0;
      for (int b = 0; b < n; ++b) s += Ginv[a * n + b] * v[b];
      u[a] = s;
    }
    double s = 0.0;
    for (int r = 0; r < m; ++r) s += poly_dot(u, n, (double)(r - h) / h) * y[base + r];
    yf[base + row] = s;
    double hd = 0.0;
    for (int a = 0; a < n; ++a) hd += u[a] * v[a];
    hsum += hd;
  }
  hsum = block_sum(hsum, red);
  __syncthreads();
  double rss = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    double r = yf[j] - y[j];
    rss += r * r;
  }
  rss = block_sum(rss, red);
  double k = (double)(N - 2 * h) * Ginv[0] + hsum;
  // filtered derivative, its target power and curvature
  double mean = 0.0;
  for (int j = threadIdx.x; j < cfg.L; j += blockDim.x) {
    int jj = cfg.i0 + j;
    double dd = (yf[jj + 1] - yf[jj - 1]) / (2.0 * cfg.dw);
    x[j] = dd;
    mean += dd;
  }
  mean = block_sum(mean, red) / cfg.L;
  __syncthreads();
  for (int j = threadIdx.x; j < cfg.L; j += blockDim.x) x[j] = hann(j, cfg.L) * (x[j] - mean);
  __syncthreads();
  double kept = 0.0;
  for (int b = 0; b < Q.nbins; ++b) kept += dft_power(x, cfg.L, Q.bins[b], red);
  double cf = 0.0;
  for (int j = 1 + threadIdx.x; j < N - 1; j += blockDim.x) {
    double d2 = yf[j + 1] - 2.0 * yf[j] + yf[j - 1];
    cf += d2 * d2;
  }
  cf = block_sum(cf, red);
  if (threadIdx.x == 0) {
    // sign changes of the filtered dS/dw over the featureless range, zeros skipped
    int sc = 0, prev = 0;
    for (int j = cfg.i0; j <= cfg.i1; ++j) {
      double dd = (yf[j + 1] - yf[j - 1]) / (2.0 * cfg.dw);
      int sg = (dd > 0.0) - (dd < 0.0);
      if (sg == 0) continue;
      if (prev != 0 && sg != prev) ++sc;
      prev = sg;
    }
    CandOut o;
    o.valid = (N - k - 1.0 > 0.0) ? 1 : 0;
    double aicc = N * log(fmax(rss, 1e-300) / N) + 2.0 * k + 2.0 * k * (k + 1.0) / (N - k - 1.0);
    double rf = Q.raw_power > 0.0 ? kept / Q.raw_power : 0.0;
    double fpen = log(fmax(rf, cfg.r0) / cfg.r0);
    double cpen = Q.curv_raw > 0.0 ? cf / Q.curv_raw : 0.0;
    o.score = aicc + cfg.lf * fpen + cfg.lc * cpen;
    o.sign_changes = sc;
    cout[(size_t)iq * cfg.ncand + ci] = o;
  }
}

struct DegOut {
  int d, m, accepted;
  double score, mean_ratio, rms_ratio;
};

// Positive branch point i: (w_i, S_i) with the S(0) point first when 0 is off the grid.
__device__ inline double branch_x(const AttCfg& c, const double* omega, int i) {
  if (c.zero) return omega[c.jp + i];
  return i == 0 ? 0.0 : omega[c.jp + i - 1];
}

__device__ inline double branch_wt(const AttCfg& c, const double* omega, int i, int npos) {
  double w = 0.0, x = branch_x(c, omega, i);
  if (i > 0) w += 0.5 * (x - branch_x(c, omega, i - 1));
  if (i < npos - 1) w += 0.5 * (branch_x(c, omega, i + 1) - x);
  return w;
}

// block per q.  best window per degree, constraints (Eqs. 5, 7), S_p.
__global__ void att_select(const double* __restrict__ S, const double2* __restrict__ s0,
                           const double* __restrict__ omega, AttCfg cfg,
                           const int2* __restrict__ cands, const double* __restrict__ yf_all,
                           const CandOut* __restrict__ cout, double* __restrict__ Fn_work,
                           double* __restrict__ Sp, DegOut* __restrict__ dout,
                           int* __restrict__ nacc_out) {
  __shared__ double red[33];
  __shared__ int chosen[kMaxDegree];
  const int iq = blockIdx.x;
  const int N = cfg.N;
  const double beta = 1.0 / cfg.T;
  const double* Sq = S + (size_t)iq * cfg.nw;
  const double* y = Sq + cfg.jp;
  const CandOut* co = cout + (size_t)iq * cfg.ncand;
  if (threadIdx.x == 0) {
    for (int di = 0; di < cfg.ndeg; ++di) {
      int d = cfg.dmin + di, best = -1;
      for (int c = 0; c < cfg.ncand; ++c) {
        if (cands[c].x != d || !co[c].valid) continue;
        if (best < 0) {
          best = c;
          continue;
        }
        double sb = co[best].score, s = co[c].score;
        bool tie = fabs(s - sb) <= 1e-9 * fabs(sb);
        bool better = (!tie && s < sb) ||
                      (tie && (co[c].sign_changes < co[best].sign_changes ||
                               (co[c].sign_changes == co[best].sign_changes && cands[c].y < cands[best].y)));
        if (better) best = c;
      }
      chosen[di] = best;
    }
  }
  __syncthreads();
  const int npos = N + (cfg.zero ? 0 : 1);
  const int off = cfg.zero ? 0 : 1;
  // reference F(beta/2)
  const double S0 = cfg.T * s0[iq].x / (M_PI * cfg.n);   // the w -> 0 limit (zerofreq.cu)
  double fr = 0.0;
  for (int i = threadIdx.x; i < npos; i += blockDim.x) {
    double xv = branch_x(cfg, omega, i);
    double sv = (i < off) ? S0 : y[i - off];
    fr += branch_wt(cfg, omega, i, npos) * sv * 2.0 * exp(-0.5 * beta * xv);
  }
  double Fref = block_sum(fr, red);
  int nacc = 0;
  double* Fn = Fn_work + (size_t)iq * cfg.ntau;
  for (int di = 0; di < cfg.ndeg; ++di) {
    int c = chosen[di];
    DegOut o;
    o.d = cfg.dmin + di;
    o.m = -1;
    o.accepted = 0;
    o.score = 0.0;
    o.mean_ratio = o.rms_ratio = 0.0;
    if (c >= 0) {
      const double* yf = yf_all + ((size_t)iq * cfg.ncand + c) * N;
      // F_n(tau) for tau on [0, beta/2]
      for (int it = threadIdx.x; it < cfg.ntau; it += blockDim.x) {
        double ta = 0.5 * beta * it / (cfg.ntau - 1);
        double acc = 0.0;
        for (int i = off; i < npos; ++i) {
          double xv = branch_x(cfg, omega, i);
          acc += branch_wt(cfg, omega, i, npos) * (y[i - off] - yf[i - off]) *
                 (exp(-ta * xv) + exp(-(beta - ta) * xv));
        }
        Fn[it] = acc;
      }
      __syncthreads();
      double dt = 0.5 * beta / (cfg.ntau - 1);
      double s1 = 0.0;
      for (int it = threadIdx.x; it < cfg.ntau; it += blockDim.x) {
        double w = (it == 0 || it == cfg.ntau - 1) ? 0.5 * dt : dt;
        s1 += w * Fn[it];
      }
      double Fbar = block_sum(s1, red) * 2.0 / beta;
      double s2 = 0.0;
      for (int it = threadIdx.x; it < cfg.ntau; it += blockDim.x) {
        double w = (it == 0 || it == cfg.ntau - 1) ? 0.5 * dt : dt;
        s2 += w * (Fn[it] - Fbar) * (Fn[it] - Fbar);
      }
      double sig = sqrt(fmax(block_sum(s2, red) * 2.0 / beta, 0.0));
      o.m = cands[c].y;
      o.score = co[c].score;
      o.mean_ratio = fabs(Fbar) / Fref;
      o.rms_ratio = sig / Fref;
      o.accepted = (o.mean_ratio <= cfg.accept_mean && o.rms_ratio <= cfg.accept_rms) ? 1 : 0;
      nacc += o.accepted;
    }
    if (threadIdx.x == 0) dout[(size_t)iq * kMaxDegree + di] = o;
    __syncthreads();
  }
  // S_p
  double* out = Sp + (size_t)iq * cfg.nw;
  int bestd = -1;
  double bests = 0.0;
  for (int di = 0; di < cfg.ndeg; ++di) {
    DegOut o = dout[(size_t)iq * kMaxDegree + di];
    if (!o.accepted) continue;
    if (bestd < 0 || o.score < bests) {
      bestd = di;
      bests = o.score;
    }
  }
  for (int j = threadIdx.x; j < cfg.nw; j += blockDim.x) {
    double v = Sq[j];
    if (j >= cfg.jp && nacc > 0) {
      int i = j - cfg.jp;
      if (cfg.average) {
        double s = 0.0;
        for (int di = 0; di < cfg.ndeg; ++di) {
          if (!dout[(size_t)iq * kMaxDegree + di].accepted) continue;
          s += yf_all[((size_t)iq * cfg.ncand + chosen[di]) * N + i];
        }
        v = s / nacc;
      } else {
        v = yf_all[((size_t)iq * cfg.ncand + chosen[bestd]) * N + i];
      }
    }
    out[j] = v;
  }
  if (threadIdx.x == 0) nacc_out[iq] = nacc;
}

// Configuration, validation and the (degree, window) candidates of one attenuation call.
lrt_status plan_attenuation(const lrt_ctx* c, const lrt_atten_params* pin, AttCfg& cfg,
                            std::vector<int2>& cands) {
  lrt_atten_params p{};
  if (pin) p = *pin;
  cfg = AttCfg{};
  cfg.jp = c->nw;
  for (int j = 0; j < c->nw; ++j)
    if (c->omega[j] >= 0.0) {
      cfg.jp = j;
      break;
    }
  cfg.N = c->nw - cfg.jp;
  if (cfg.N < 8) {
    set_error("attenuation needs at least 8 samples with w >= 0");
    return LRT_EINVAL;
  }
  cfg.zero = c->omega[cfg.jp] == 0.0;
  cfg.dw = c->omega[cfg.jp + 1] - c->omega[cfg.jp];
  for (int j = cfg.jp + 1; j < c->nw; ++j)
    if (std::fabs((c->omega[j] - c->omega[j - 1]) - cfg.dw) > 1e-9 * cfg.dw) {
      set_error("attenuation needs uniformly spaced samples with w >= 0");
      return LRT_EINVAL;
    }
  const int N = cfg.N;
  if (p.feat_lo <= 0.0 && p.feat_hi <= 0.0) {
    cfg.i0 = std::max(1, (int)std::floor(0.05 * (N - 1)));
    cfg.i1 = std::min(N - 2, (int)std::ceil(0.95 * (N - 1)));
  } else {
    const double* w = c->omega.data() + cfg.jp;
    cfg.i0 = std::max(1, (int)(std::lower_bound(w, w + N, p.feat_lo) - w));
    cfg.i1 = std::min(N - 2, (int)(std::upper_bound(w, w + N, p.feat_hi) - w) - 1);
  }
  cfg.L = cfg.i1 - cfg.i0 + 1;
  if (cfg.L < 8) {
    set_error("featureless range too short");
    return LRT_EINVAL;
  }
  cfg.K = cfg.L / 2;
  double low = p.low_exclude > 0 ? p.low_exclude : 0.05;
  cfg.kmin = std::max(1, (int)std::ceil(low * cfg.K));
  cfg.ntargets = p.n_targets > 0 ? std::min(p.n_targets, kMaxTargets) : 2;
  cfg.lf = p.lambda_f > 0 ? p.lambda_f : N;
  cfg.lc = p.lambda_c > 0 ? p.lambda_c : N;
  cfg.r0 = p.retain_floor > 0 ? p.retain_floor : 1e-4;
  cfg.dmin = p.d_min > 0 ? p.d_min : 1;
  int dmax = p.d_max > 0 ? p.d_max : 4;
  if (dmax < cfg.dmin || dmax - cfg.dmin + 1 > kMaxDegree || dmax > kMaxDegree) {
    set_error("degree range");
    return LRT_EINVAL;
  }
  cfg.ndeg = dmax - cfg.dmin + 1;
  cfg.ntau = p.ntau > 1 ? p.ntau : 64;
  cfg.accept_mean = p.accept_mean > 0 ? p.accept_mean : 4e-3;
  cfg.accept_rms = p.accept_rms > 0 ? p.accept_rms : 4.2e-5;
  cfg.average = (p.average == 2) ? 0 : 1;
  cfg.T = c->T;
  cfg.n = c->density;
  cfg.nw = c->nw;
  // window grid: m = 2 round(w / (2 dw)) + 1 over linspace(w_min, w_max, n_w), distinct,
  // ascending; candidates with d + 2 <= m <= N
  double wlo = p.w_min > 0 ? p.w_min : 4.0 * cfg.dw;
  double whi = p.w_max > 0 ? p.w_max : 0.25 * N * cfg.dw;
  int nwin = p.n_w > 0 ? p.n_w : 24;
  std::set<int> ms;
  for (int i = 0; i < nwin; ++i) {
    double w = nwin == 1 ? wlo : wlo + (whi - wlo) * i / (nwin - 1);
    ms.insert(2 * (int)std::floor(w / (2.0 * cfg.dw) + 0.5) + 1);
  }
  cands.clear();
  for (int d = cfg.dmin; d <= dmax; ++d)
    for (int m : ms)
      if (m >= d + 2 && m <= N && m >= 3) cands.push_back(make_int2(d, m));
  cfg.ncand = (int)cands.size();
  if (cfg.ncand == 0) {
    set_error("no admissible (degree, window) candidate");
    return LRT_EINVAL;
  }
  return LRT_OK;
}

// Byte offsets of the workspace parts (each rounded up to 256 bytes).
struct AttLayout {
  size_t prep, yf, dwork, fnw, spd, aq, co, dout, dc, nacc, total;
};
AttLayout attenuation_layout(const AttCfg& cfg, int nq) {
  auto up = [](size_t n) { return (n + 255) / 256 * 256; };
  const size_t sz[10] = {up((size_t)nq * (cfg.L + cfg.K + 1) * sizeof(double)),
                         up((size_t)nq * cfg.ncand * cfg.N * sizeof(double)),
                         up((size_t)nq * cfg.ncand * cfg.L * sizeof(double)),
                         up((size_t)nq * cfg.ntau * sizeof(double)),
                         up((size_t)nq * cfg.nw * sizeof(double)),
                         up(nq * sizeof(AttQ)),
                         up((size_t)nq * cfg.ncand * sizeof(CandOut)),
                         up((size_t)nq * kMaxDegree * sizeof(DegOut)),
                         up(cfg.ncand * sizeof(int2)),
                         up(nq * sizeof(int))};
  size_t off[10], o = 0;
  for (int i = 0; i < 10; ++i) {
    off[i] = o;
    o += sz[i];
  }
  return AttLayout{off[0], off[1], off[2], off[3], off[4], off[5], off[6], off[7], off[8], off[9], o};
}

// The kernels of one attenuation call on the workspace at buf (laid out by attenuation_layout),
// then S_p and the report to the host.
lrt_status run_on_workspace(const lrt_ctx* c, const AttCfg& cfg, const std::vector<int2>& cands,
                            char* buf, const double* S_dev, const double2* s0_dev, int rows,
                            double* Sp_host, lrt_atten_report* rep, cudaStream_t s) {
  const int nq = rows;   // spectrum rows: (q, eta) pairs of the context, or the caller's
  const AttLayout L = attenuation_layout(cfg, nq);
  double* prep = (double*)(buf + L.prep);
  double* yf = (double*)(buf + L.yf);
  double* dwork = (double*)(buf + L.dwork);
  double* fnw = (double*)(buf + L.fnw);
  double* spd = (double*)(buf + L.spd);
  AttQ* aq = (AttQ*)(buf + L.aq);
  CandOut* co = (CandOut*)(buf + L.co);
  DegOut* dout = (DegOut*)(buf + L.dout);
  int2* dc = (int2*)(buf + L.dc);
  int* nacc = (int*)(buf + L.nacc);
  LRT_CUDA(cudaMemcpyAsync(dc, cands.data(), cands.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
  att_prep<<<nq, 256, 0, s>>>(S_dev, cfg, prep, aq);
  LRT_CUDA(cudaGetLastError());
  att_candidates<<<dim3(cfg.ncand, nq), 256, 0, s>>>(S_dev, cfg, dc, aq, yf, dwork, co);
  LRT_CUDA(cudaGetLastError());
  att_select<<<nq, 256, 0, s>>>(S_dev, s0_dev, c->dw.omega, cfg, dc, yf, co, fnw, spd, dout, nacc);
  count_launch(c, 3);
  LRT_CUDA(cudaGetLastError());
  LRT_CUDA(cudaMemcpyAsync(Sp_host, spd, (size_t)nq * c->nw * sizeof(double), cudaMemcpyDeviceToHost, s));
  std::vector<AttQ> hq(nq);
  std::vector<DegOut> hd((size_t)nq * kMaxDegree);
  std::vector<int> hn(nq);
  LRT_CUDA(cudaMemcpyAsync(hq.data(), aq, nq * sizeof(AttQ), cudaMemcpyDeviceToHost, s));
  LRT_CUDA(cudaMemcpyAsync(hd.data(), dout, hd.size() * sizeof(DegOut), cudaMemcpyDeviceToHost, s));
  LRT_CUDA(cudaMemcpyAsync(hn.data(), nacc, nq * sizeof(int), cudaMemcpyDeviceToHost, s));
  LRT_CUDA(cudaStreamSynchronize(s));
  if (rep) {
    for (int iq = 0; iq < nq; ++iq) {
      lrt_atten_report& r = rep[iq];
      r.n_accepted = hn[iq];
      for (int i = 0; i < 4; ++i) r.targets[i] = i < hq[iq].ntg ? hq[iq].tg[i] : -1;
      for (int i = 0; i < LRT_ATTEN_MAX_DEG; ++i) {
        if (i < cfg.ndeg && hd[(size_t)iq * kMaxDegree + i].m > 0) {
          const DegOut& o = hd[(size_t)iq * kMaxDegree + i];
          r.degree[i] = o.d;
          r.window[i] = o.m;
          r.score[i] = o.score;
          r.mean_ratio[i] = o.mean_ratio;
          r.rms_ratio[i] = o.rms_ratio;
          r.accepted[i] = o.accepted;
        } else {
          r.degree[i] = -1;
          r.window[i] = 0;
          r.score[i] = r.mean_ratio[i] = r.rms_ratio[i] = 0.0;
          r.accepted[i] = 0;
        }
      }
    }
  }
  return LRT_OK;
}

}  // namespace

lrt_status run_attenuation_rows(const lrt_ctx* c, const lrt_atten_params* pin, const double* S_dev,
                                const double2* s0_dev, int rows, double* Sp_host,
                                lrt_atten_report* rep, cudaStream_t s) {
  AttCfg cfg;
  std::vector<int2> cands;
  LRT_TRY(plan_attenuation(c, pin, cfg, cands));
  const AttLayout L = attenuation_layout(cfg, rows);
  char* buf = nullptr;
  LRT_CUDA(cudaMalloc(&buf, L.total));
  struct Free {
    char* b;
    ~Free() { cudaFree(b); }
  } fr{buf};
  return run_on_workspace(c, cfg, cands, buf, S_dev, s0_dev, rows, Sp_host, rep, s);
}

lrt_status run_attenuation(const lrt_ctx* c, const lrt_atten_params* pin, const double* S_dev,
                           double* Sp_host, lrt_atten_report* rep, cudaStream_t s) {
  return run_attenuation_rows(c, pin, S_dev, c->dw.s0, nrow(c), Sp_host, rep, s);
}

// ---------------------------------------------------------------------------------------
// Allocation-free attenuation.  The workspace is one file-scope device array that every GPU
// loading the library holds until the process exits; its device address is looked up once
// per device (cudaGetSymbolAddress with that device current) on the first call made for a
// context on that device.  Calls share the array: two calls whose kernels overlap on the GPU
// (from different host threads or streams) race and corrupt each other's results.
// The paper has no counterpart: this entry point exists for callers that cannot allocate
// device memory at call time.
constexpr size_t kNoAllocScratchBytes = 16u << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_atten_scratch[kNoAllocScratchBytes];

static std::mutex g_scratch_mu;
static void* g_scratch_addr[64] = {};

static lrt_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal out of range for the fixed workspace table");
    return LRT_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_atten_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress for the attenuation workspace: ") +
                cudaGetErrorString(e));
      return LRT_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return LRT_OK;
}

lrt_status run_attenuation_noalloc(const lrt_ctx* c, const lrt_atten_params* pin,
                                   const double* S_dev, double* Sp_host, lrt_atten_report* rep,
                                   cudaStream_t s) {
  AttCfg cfg;
  std::vector<int2> cands;
  LRT_TRY(plan_attenuation(c, pin, cfg, cands));
  const size_t need = attenuation_layout(cfg, nrow(c)).total;
  if (need > kNoAllocScratchBytes) {
    set_error("attenuation workspace of " + std::to_string(need) + " bytes exceeds the " +
              std::to_string(kNoAllocScratchBytes) +
              "-byte fixed array of the allocation-free entry point (fewer q, windows or "
              "frequencies per call fit)");
    return LRT_EINVAL;
  }
  void* base = nullptr;
  LRT_TRY(scratch_address(c->device, &base));
  // the array keeps the previous call's contents: start this call from zeros
  LRT_CUDA(cudaMemsetAsync(base, 0, need, s));
  return run_on_workspace(c, cfg, cands, static_cast<char*>(base), S_dev, c->dw.s0, nrow(c), Sp_host,
                          rep, s);
}

}  // namespace lrt

// Allocation-free variant of lrtddft_attenuate (declared in include/lrtddft.h).
extern "C" lrt_status lrtddft_attenuate_noalloc(lrt_ctx* c, const lrt_atten_params* p, double* Sp,
                                                lrt_atten_report* rep) {
  using namespace lrt;
  if (!c || !Sp) {
    set_error("NULL argument");
    return LRT_EINVAL;
  }
  if (c->host_only) {
    set_error("host-only context");
    return LRT_ESTATE;
  }
  LRT_CUDA(cudaSetDevice(c->device));
  for (auto& Q : c->qd)
    if (!Q.have_chi) {
      set_error("spectra requested before dyson_solve on every q");
      return LRT_ESTATE;
    }
  LRT_CUDA(cudaDeviceSynchronize());
  LRT_TRY(launch_dsf(c, c->dw.S, 0));
  LRT_TRY(run_attenuation_noalloc(c, p, c->dw.S, Sp, rep, 0));
  return check_status_word(c);
}
