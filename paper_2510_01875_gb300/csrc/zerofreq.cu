// The w -> 0 limit of the fluctuation-dissipation relation (Eq. 8) and its tangents.
//
// S(q,0) = lim_{w->0} -Im chi_00(w) / (pi n (1 - e^{-w/T})) = -(T/(pi n)) d Im chi_00/dw at 0
// (Im chi_00(0) = 0 on the time-reversal-symmetric pair meshes).  chi0 depends on w and eta only
// through w + i eta and K depends on neither, so chi_00 is analytic in w + i eta and
// d chi_00/dw = -i d chi_00/d eta:
//   S(q,0) = (T/(pi n)) Re s,   s = d chi_00/d eta at w = 0 = u^T E v,
//   E = d chi0/d eta = (2/(N_k Omega)) sum_p rho_p rho_p^* (-i df_p)/(Delta_p + i eta)^2,
//   M = 1 - chi0(0) K,  M x = chi0_{:,0},  M^T u = e_0,  v = K x + e_0,
// so s = pref sum_p (u . rho_p)(rho_p^* . v)(-i df_p)/(Delta_p + i eta)^2: a projection over the
// pairs (2 N_G complex MACs each), run right after the contraction of the q while its pair
// densities are resident.
//
// Tangents of s (the adjoint of S(0)); all dot products are bilinear (no conjugation):
//   a_th = (d chi0/d th)^T u,  b_th = (d chi0/d th) v  (th = T, eta; zero for A, B, C),
//   e_th = u^T (dE/d th) v,  dE/dT = sum rho rho^* (-i d df_p/dT)/(...)^2,
//                            dE/deta = sum rho rho^* (-2 df_p)/(...)^3,
//   y = M^{-1} b_eta,  z = M^{-T} (K a_eta),
//   ds/d th = r_th . y + e_th + a_eta . (dK_th x) + z . s_th,
//   r_th = K a_th + dK_th (chi0^T u),  s_th = b_th + chi0 (dK_th x).
// (From s = u^T E v: du = M^{-T} r_th, dv = dK x + K dx, dx = M^{-1} s_th.)
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "lrt_internal.h"

namespace lrt {
namespace {

__device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ inline double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ inline void csub(double2& a, double2 b) {
  a.x -= b.x;
  a.y -= b.y;
}

constexpr int kThreads = 256;

// One block: LU with partial pivoting (rows swapped in full, multipliers kept below the
// diagonal, P M = L U) of M = 1 - X K, X = chi0 at one frequency ([N][N], row-major), then
//   M out_n = rhs_n  (rhs_n NULL: X column 0),
//   M^T out_t = tscale * rhs_t  (rhs_t NULL: e_0; tscale NULL: 1),
// and, when v_out is given, v_out = K out_n + e_0.  GM: the matrix in ws (N x (N + 1)).
template <bool GM>
__global__ void __launch_bounds__(kThreads) lu_two_solves(
    const double2* __restrict__ X, const double* __restrict__ K, int N,
    const double2* __restrict__ rhs_n, const double2* __restrict__ rhs_t,
    const double* __restrict__ tscale, double2* __restrict__ out_n, double2* __restrict__ out_t,
    double2* __restrict__ v_out, int* __restrict__ status, double2* ws) {
  extern __shared__ double2 sm[];
  const int ld = N + 1;
  double2* A = GM ? ws : sm;
  double2* bn = GM ? sm : sm + (size_t)N * ld;
  double2* bt = bn + N;
  double2* fac = bt + N;
  int* piv = reinterpret_cast<int*>(fac + N);
  __shared__ int piv_s, bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) bad = 0;
  for (int e = tid; e < N * N; e += nt) {
    const int r = e / N, j = e % N;
    const double2 v = X[e];
    double2 m = make_double2(-v.x * K[j], -v.y * K[j]);
    if (r == j) m.x += 1.0;
    A[r * ld + j] = m;
  }
  for (int r = tid; r < N; r += nt) {
    bn[r] = rhs_n ? rhs_n[r] : X[(size_t)r * N];
    double2 t = rhs_t ? rhs_t[r] : make_double2(r == 0 ? 1.0 : 0.0, 0.0);
    if (rhs_t && tscale) t = make_double2(t.x * tscale[r], t.y * tscale[r]);
    bt[r] = t;
  }
  __syncthreads();
  for (int c = 0; c < N; ++c) {
    if (tid < 32) {
      double best = -1.0;
      int bi = c;
      for (int r = c + tid; r < N; r += 32) {
        const double2 v = A[r * ld + c];
        const double a = v.x * v.x + v.y * v.y;
        if (a > best) {
          best = a;
          bi = r;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) {
        piv_s = bi;
        piv[c] = bi;
        if (!(best > 0.0)) bad = 1;
      }
    }
    __syncthreads();
    const int p = piv_s;
    if (p != c) {
      for (int j = tid; j < N; j += nt) {
        const double2 t = A[c * ld + j];
        A[c * ld + j] = A[p * ld + j];
        A[p * ld + j] = t;
      }
      if (tid == 0) {
        const double2 t = bn[c];
        bn[c] = bn[p];
        bn[p] = t;
      }
    }
    __syncthreads();
    const double2 d = A[c * ld + c];
    for (int r = c + 1 + tid; r < N; r += nt) fac[r] = cdiv(A[r * ld + c], d);
    __syncthreads();
    const int rows = N - c - 1, cols = N - c;   // columns c+1..N-1 plus the right-hand side
    for (int e = tid; e < rows * cols; e += nt) {
      const int r = c + 1 + e / cols, jj = e % cols;
      const double2 f = fac[r];
      if (jj == cols - 1)
        csub(bn[r], cmul(f, bn[c]));
      else
        csub(A[r * ld + c + 1 + jj], cmul(f, A[c * ld + c + 1 + jj]));
    }
    __syncthreads();
    for (int r = c + 1 + tid; r < N; r += nt) A[r * ld + c] = fac[r];   // L below the diagonal
    __syncthreads();
  }
  // U out_n = bn (column oriented)
  for (int c = N - 1; c >= 0; --c) {
    if (tid == 0) bn[c] = cdiv(bn[c], A[c * ld + c]);
    __syncthreads();
    const double2 xc = bn[c];
    for (int r = tid; r < c; r += nt) csub(bn[r], cmul(A[r * ld + c], xc));
    __syncthreads();
  }
  // M^T = U^T L^T P:  U^T w = bt (forward), L^T w' = w (backward, unit diagonal), out = P^T w'
  for (int c = 0; c < N; ++c) {
    if (tid == 0) bt[c] = cdiv(bt[c], A[c * ld + c]);
    __syncthreads();
    const double2 wc = bt[c];
    for (int r = c + 1 + tid; r < N; r += nt) csub(bt[r], cmul(A[c * ld + r], wc));
    __syncthreads();
  }
  for (int c = N - 1; c >= 0; --c) {
    const double2 wc = bt[c];
    for (int r = tid; r < c; r += nt) csub(bt[r], cmul(A[c * ld + r], wc));
    __syncthreads();
  }
  if (tid == 0)
    for (int c = N - 1; c >= 0; --c) {
      const int p = piv[c];
      if (p != c) {
        const double2 t = bt[c];
        bt[c] = bt[p];
        bt[p] = t;
      }
    }
  __syncthreads();
  for (int r = tid; r < N; r += nt) {
    out_n[r] = bn[r];
    out_t[r] = bt[r];
    if (v_out) v_out[r] = make_double2(K[r] * bn[r].x + (r == 0 ? 1.0 : 0.0), K[r] * bn[r].y);
  }
  if (tid == 0 && bad) atomicOr(status, 1);
}

// Pair densities of pair p at G, either layout: blocked FP32 [p/32][gpad][32] (split path) or
// FP64 [G][ld].
template <typename R2>
__device__ inline double2 rho_at(const R2* rho, long long ld, int gpad, long long p, int G);
template <>
__device__ inline double2 rho_at<float2>(const float2* rho, long long, int gpad, long long p, int G) {
  const float2 v = rho[((size_t)((p >> 5) * gpad + G) << 5) + (size_t)(p & 31)];
  return make_double2(v.x, v.y);
}
template <>
__device__ inline double2 rho_at<double2>(const double2* rho, long long ld, int, long long p, int G) {
  return rho[(size_t)G * ld + (size_t)p];
}

// s = scale sum_p (u . rho_p)(rho_p^* . v)(-i df_p)/(Delta_p + i eta)^2 over all pairs, one
// thread per pair (consecutive lanes on consecutive pairs, so every G row is read coalesced).
// Split path: FP32 pair densities, Delta = Delta_hi + Delta_lo and df (times sB) from the
// contraction's float4 pair weights, FP32 products and per-thread partial sums; FP64 path:
// FP64 throughout.  The partial sums are reduced in FP64 and added into *out.
template <bool SPLIT>
__global__ void __launch_bounds__(kThreads) s0_project(
    const void* __restrict__ rho_v, long long ld, int gpad, int N, const double2* __restrict__ u,
    const double2* __restrict__ v, const float4* __restrict__ pw, const double* __restrict__ delta,
    const double* __restrict__ df, long long np, double eta, double scale, double2* __restrict__ out) {
  using R = typename std::conditional<SPLIT, float, double>::type;
  extern __shared__ unsigned char smraw[];
  R* us = reinterpret_cast<R*>(smraw);   // [N][2]
  R* vs = us + 2 * N;                    // [N][2]
  for (int g = threadIdx.x; g < N; g += blockDim.x) {
    us[2 * g] = (R)u[g].x;
    us[2 * g + 1] = (R)u[g].y;
    vs[2 * g] = (R)v[g].x;
    vs[2 * g + 1] = (R)v[g].y;
  }
  __syncthreads();
  const R e = (R)eta;
  R accr = 0, acci = 0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    R ar = 0, ai = 0, br = 0, bi = 0;
    for (int g = 0; g < N; ++g) {
      R rr, ri;
      if (SPLIT) {
        const float2 t = static_cast<const float2*>(rho_v)[((size_t)((p >> 5) * gpad + g) << 5) + (size_t)(p & 31)];
        rr = t.x;
        ri = t.y;
      } else {
        const double2 t = static_cast<const double2*>(rho_v)[(size_t)g * ld + (size_t)p];
        rr = (R)t.x;
        ri = (R)t.y;
      }
      const R ur = us[2 * g], ui = us[2 * g + 1], vr = vs[2 * g], vi = vs[2 * g + 1];
      ar += ur * rr - ui * ri;   // a += u rho
      ai += ur * ri + ui * rr;
      br += rr * vr + ri * vi;   // b += conj(rho) v
      bi += rr * vi - ri * vr;
    }
    R x, f;
    if (SPLIT) {
      const float4 w = pw[p];
      x = w.x + w.y;
      f = w.z;
    } else {
      x = (R)delta[p];
      f = (R)df[p];
    }
    const R d2 = x * x + e * e;
    const R inv2 = (R)1 / (d2 * d2);
    // -i df/(x + i e)^2 = df (-2 x e - i (x^2 - e^2)) / |x + i e|^4
    const R qr = -(R)2 * f * x * e * inv2, qi = -f * (x * x - e * e) * inv2;
    const R tr = ar * br - ai * bi, ti = ar * bi + ai * br;
    accr += tr * qr - ti * qi;
    acci += tr * qi + ti * qr;
  }
  double sr = (double)accr, si = (double)acci;
  for (int off = 16; off > 0; off >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, off);
    si += __shfl_down_sync(0xffffffffu, si, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out->x, scale * sr);
    atomicAdd(&out->y, scale * si);
  }
}

constexpr int ZCH = 32;   // pairs per chunk of the vector projections

// Second-order pieces at w = 0 (FP64 arithmetic, either pair-density layout), scaled by `scale`
// and added into vec[4][N] = (a_T, a_eta, b_T, b_eta) and sc[2] = (e_T, e_eta):
//   a_th[G'] = sum_p (u . rho_p) rho_p^*(G') dw_th,  b_th[G] = sum_p rho_p(G) (rho_p^* . v) dw_th,
//   dw_T = d df/dT / z,  dw_eta = -i df / z^2,  z = Delta + i eta,
//   e_T = sum_p a_p b_p (-i d df/dT) / z^2,  e_eta = sum_p a_p b_p (-2 df) / z^3.
template <typename R2>
__global__ void __launch_bounds__(kThreads) zf_vector_project(
    const R2* __restrict__ rho, long long ld, int gpad, int N, const double2* __restrict__ u,
    const double2* __restrict__ v, const double* __restrict__ delta, const double* __restrict__ df,
    const double* __restrict__ ddf, long long np, long long per_block, double eta, double scale,
    double2* __restrict__ vec, double2* __restrict__ sc) {
  extern __shared__ double2 zs[];
  double2* rs = zs;                        // [N][ZCH]
  double2* acc = rs + (size_t)N * ZCH;     // [4][N]
  double2* us = acc + 4 * (size_t)N;       // [N]
  double2* vs = us + N;                    // [N]
  __shared__ double2 part[8][ZCH][2];
  __shared__ double2 coef[4][ZCH];
  __shared__ double2 scs[2];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  for (int g = tid; g < N; g += blockDim.x) {
    us[g] = u[g];
    vs[g] = v[g];
    for (int j = 0; j < 4; ++j) acc[j * N + g] = make_double2(0, 0);
  }
  if (tid < 2) scs[tid] = make_double2(0, 0);
  const long long pb = (long long)blockIdx.x * per_block, pe = min(np, pb + per_block);
  for (long long p0 = pb; p0 < pe; p0 += ZCH) {
    __syncthreads();
    for (int e2 = tid; e2 < N * ZCH; e2 += blockDim.x) {
      const int g = e2 / ZCH, l = e2 % ZCH;
      const long long p = p0 + l;
      rs[e2] = p < pe ? rho_at<R2>(rho, ld, gpad, p, g) : make_double2(0, 0);
    }
    __syncthreads();
    // a_p and b_p: warp wp sums G = wp, wp + 8, ... for pair lane
    double2 a = make_double2(0, 0), b = make_double2(0, 0);
    for (int g = wp; g < N; g += 8) {
      const double2 r = rs[g * ZCH + lane];
      const double2 t1 = cmul(us[g], r);
      a.x += t1.x;
      a.y += t1.y;
      const double2 t2 = cmul(make_double2(r.x, -r.y), vs[g]);
      b.x += t2.x;
      b.y += t2.y;
    }
    part[wp][lane][0] = a;
    part[wp][lane][1] = b;
    __syncthreads();
    if (wp == 0) {
      double2 A = make_double2(0, 0), B = make_double2(0, 0);
      for (int k = 0; k < 8; ++k) {
        A.x += part[k][lane][0].x;
        A.y += part[k][lane][0].y;
        B.x += part[k][lane][1].x;
        B.y += part[k][lane][1].y;
      }
      const long long p = p0 + lane;
      double2 wT = make_double2(0, 0), wE = make_double2(0, 0), sT = make_double2(0, 0),
              sE = make_double2(0, 0);
      if (p < pe) {
        const double2 z = make_double2(delta[p], eta);
        const double2 iz = cdiv(make_double2(1, 0), z);
        const double2 iz2 = cmul(iz, iz), iz3 = cmul(iz2, iz);
        const double f = df[p], g = ddf[p];
        wT = make_double2(g * iz.x, g * iz.y);                        // d df/dT / z
        wE = cmul(make_double2(0, -f), iz2);                          // -i df / z^2
        const double2 ab = cmul(A, B);
        sT = cmul(ab, cmul(make_double2(0, -g), iz2));                // -i d df/dT / z^2
        sE = cmul(ab, make_double2(-2.0 * f * iz3.x, -2.0 * f * iz3.y));   // -2 df / z^3
      }
      coef[0][lane] = cmul(A, wT);
      coef[1][lane] = cmul(A, wE);
      coef[2][lane] = cmul(B, wT);
      coef[3][lane] = cmul(B, wE);
      for (int off = 16; off > 0; off >>= 1) {
        sT.x += __shfl_down_sync(0xffffffffu, sT.x, off);
        sT.y += __shfl_down_sync(0xffffffffu, sT.y, off);
        sE.x += __shfl_down_sync(0xffffffffu, sE.x, off);
        sE.y += __shfl_down_sync(0xffffffffu, sE.y, off);
      }
      if (lane == 0) {
        scs[0].x += sT.x;
        scs[0].y += sT.y;
        scs[1].x += sE.x;
        scs[1].y += sE.y;
      }
    }
    __syncthreads();
    for (int g = tid; g < N; g += blockDim.x) {
      double2 s0 = acc[g], s1 = acc[N + g], s2 = acc[2 * N + g], s3 = acc[3 * N + g];
      for (int l = 0; l < ZCH; ++l) {
        const double2 r = rs[g * ZCH + l];
        const double2 rc = make_double2(r.x, -r.y);
        const double2 t0 = cmul(rc, coef[0][l]), t1 = cmul(rc, coef[1][l]);
        const double2 t2 = cmul(r, coef[2][l]), t3 = cmul(r, coef[3][l]);
        s0.x += t0.x; s0.y += t0.y;
        s1.x += t1.x; s1.y += t1.y;
        s2.x += t2.x; s2.y += t2.y;
        s3.x += t3.x; s3.y += t3.y;
      }
      acc[g] = s0;
      acc[N + g] = s1;
      acc[2 * N + g] = s2;
      acc[3 * N + g] = s3;
    }
  }
  __syncthreads();
  for (int e2 = tid; e2 < 4 * N; e2 += blockDim.x) {
    atomicAdd(&vec[e2].x, scale * acc[e2].x);
    atomicAdd(&vec[e2].y, scale * acc[e2].y);
  }
  if (tid < 2) {
    atomicAdd(&sc[tid].x, scale * scs[tid].x);
    atomicAdd(&sc[tid].y, scale * scs[tid].y);
  }
}

__device__ double2 block_sum2(double2 v, double2* red) {
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, off);
    v.y += __shfl_down_sync(0xffffffffu, v.y, off);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double2 s = make_double2(0, 0);
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
    s.x += red[i].x;
    s.y += red[i].y;
  }
  return s;
}

// ds[5] = d s/d(T, eta, A, B, C) from the pieces above (one block).
__global__ void __launch_bounds__(kThreads) zf_combine(
    const double2* __restrict__ X, const double* __restrict__ K, const double* __restrict__ dK,
    const double2* __restrict__ x, const double2* __restrict__ u, const double2* __restrict__ vec,
    const double2* __restrict__ sc, const double2* __restrict__ y, const double2* __restrict__ z,
    int N, double2* __restrict__ ds) {
  __shared__ double2 red[kThreads / 32];
  const double2* aT = vec;
  const double2* aE = vec + N;
  const double2* bT = vec + 2 * N;
  const double2* bE = vec + 3 * N;
  // T and eta: r = K a_th, s_th = b_th
  double2 tT = make_double2(0, 0), tE = make_double2(0, 0);
  double2 tk[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  for (int g = threadIdx.x; g < N; g += blockDim.x) {
    const double2 yy = y[g], zz = z[g];
    double2 t = cmul(make_double2(K[g] * aT[g].x, K[g] * aT[g].y), yy);
    double2 t2 = cmul(zz, bT[g]);
    tT.x += t.x + t2.x;
    tT.y += t.y + t2.y;
    t = cmul(make_double2(K[g] * aE[g].x, K[g] * aE[g].y), yy);
    t2 = cmul(zz, bE[g]);
    tE.x += t.x + t2.x;
    tE.y += t.y + t2.y;
    // A, B, C: dK_j (chi0^T u) . y + a_eta . (dK_j x) + z . chi0 (dK_j x)
    double2 ct = make_double2(0, 0), m[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    for (int h = 0; h < N; ++h) {
      const double2 t3 = cmul(u[h], X[(size_t)h * N + g]);   // (chi0^T u)_g
      ct.x += t3.x;
      ct.y += t3.y;
      const double2 xh = X[(size_t)g * N + h];
      for (int j = 0; j < 3; ++j) {
        const double2 t4 = cmul(xh, make_double2(dK[j * N + h] * x[h].x, dK[j * N + h] * x[h].y));
        m[j].x += t4.x;
        m[j].y += t4.y;
      }
    }
    for (int j = 0; j < 3; ++j) {
      const double kj = dK[j * N + g];
      const double2 t5 = cmul(make_double2(kj * ct.x, kj * ct.y), yy);
      const double2 t6 = cmul(aE[g], make_double2(kj * x[g].x, kj * x[g].y));
      const double2 t7 = cmul(zz, m[j]);
      tk[j].x += t5.x + t6.x + t7.x;
      tk[j].y += t5.y + t6.y + t7.y;
    }
  }
  const double2 sT = block_sum2(tT, red);
  const double2 sE = block_sum2(tE, red);
  double2 sk[3];
  for (int j = 0; j < 3; ++j) sk[j] = block_sum2(tk[j], red);
  if (threadIdx.x == 0) {
    ds[0] = make_double2(sT.x + sc[0].x, sT.y + sc[0].y);
    ds[1] = make_double2(sE.x + sc[1].x, sE.y + sc[1].y);
    for (int j = 0; j < 3; ++j) ds[2 + j] = sk[j];
  }
}

size_t lu_smem(int N, bool gm) {
  const size_t vecs = 3 * (size_t)N * sizeof(double2) + (size_t)N * sizeof(int);
  return gm ? vecs : (size_t)N * (N + 1) * sizeof(double2) + vecs;
}

}  // namespace

// Solve M out_n = rhs_n and M^T out_t = tscale rhs_t at internal frequency w of q (defaults as
// in lu_two_solves), v_out = K out_n + e_0 if given.
lrt_status launch_lu_two_solves(const lrt_ctx* c, const QData& q, int w, const double2* rhs_n,
                                const double2* rhs_t, const double* tscale, double2* out_n,
                                double2* out_t, double2* v_out, cudaStream_t s) {
  const int N = q.nG;
  const double2* X = q.chi0 + (size_t)w * N * N;
  lrt_ctx* cc = const_cast<lrt_ctx*>(c);
  if (lu_smem(N, false) > 227 * 1024) {
    const size_t mat = (size_t)N * (N + 1) * sizeof(double2);
    if (cc->dw.zf_ws_bytes < mat) {
      // allocated by the first call that needs it (before any graph capture: the capture
      // follows an ordinary pass)
      cudaFree(cc->dw.zf_ws);
      cc->dw.zf_ws = nullptr;
      cc->dw.zf_ws_bytes = 0;
      LRT_CUDA(cudaMalloc(&cc->dw.zf_ws, mat));
      cc->dw.zf_ws_bytes = mat;
    }
    lu_two_solves<true><<<1, kThreads, lu_smem(N, true), s>>>(
        X, q.Kdev, N, rhs_n, rhs_t, tscale, out_n, out_t, v_out, c->dw.status, (double2*)cc->dw.zf_ws);
  } else {
    const size_t smem = lu_smem(N, false);
    int dev = 0;
    LRT_CUDA(cudaGetDevice(&dev));
    static size_t attr_set[64] = {0};
    if (dev < 0 || dev >= 64 || attr_set[dev] < smem) {
      LRT_CUDA(cudaFuncSetAttribute(lu_two_solves<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
      if (dev >= 0 && dev < 64) attr_set[dev] = smem;
    }
    lu_two_solves<false><<<1, kThreads, smem, s>>>(X, q.Kdev, N, rhs_n, rhs_t, tscale, out_n, out_t,
                                                   v_out, c->dw.status, nullptr);
  }
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  return LRT_OK;
}

// Zero-frequency workspace of the context (x, u, v of the forward step; the adjoint's pieces).
lrt_status ensure_zf(lrt_ctx* c) {
  if (c->dw.zf) return LRT_OK;
  const size_t n = (size_t)12 * c->nGmax + 16;
  LRT_CUDA(cudaMalloc(&c->dw.zf, n * sizeof(double2)));
  LRT_CUDA(cudaMalloc(&c->dw.s0, (size_t)nrow(c) * sizeof(double2)));
  LRT_CUDA(cudaMemset(c->dw.s0, 0, (size_t)nrow(c) * sizeof(double2)));
  return LRT_OK;
}

lrt_status launch_s0_eta(const lrt_ctx* c, const QData& q, int iq, int j, const void* rho,
                         const float4* pw, float sB, cudaStream_t s);

// s of q iq into dw.s0[iq neta ...] for every eta of the list, from this q's chi0 (already
// assembled) and pair densities: split
// path (blocked FP32 rho, float4 pair weights with df scaled by sB) or FP64 path (dw.rho,
// dw.delta, dw.df).
lrt_status launch_s0(const lrt_ctx* c, const QData& q, int iq, const void* rho, const float4* pw,
                     float sB, cudaStream_t s) {
  for (int j = 0; j < c->neta; ++j) LRT_TRY(launch_s0_eta(c, q, iq, j, rho, pw, sB, s));
  return LRT_OK;
}

// s of q iq at eta j of the eta list into dw.s0[iq neta + j]
lrt_status launch_s0_eta(const lrt_ctx* c, const QData& q, int iq, int j, const void* rho,
                         const float4* pw, float sB, cudaStream_t s) {
  const int N = q.nG;
  double2* x = c->dw.zf;
  double2* u = x + N;
  double2* v = u + N;
  double2* out = c->dw.s0 + (size_t)iq * c->neta + j;
  LRT_TRY(launch_lu_two_solves(c, q, j * c->nwi + c->hcol, nullptr, nullptr, nullptr, x, u, v, s));
  LRT_CUDA(cudaMemsetAsync(out, 0, sizeof(double2), s));
  int dev = 0, nsm = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const bool split = c->precision != LRT_PREC_FP64;
  const size_t smem = 4 * (size_t)N * (split ? sizeof(float) : sizeof(double));
  const double pref = 2.0 / (c->nk * c->volume);
  const long long blocks = std::min<long long>(4LL * nsm, (c->np + kThreads - 1) / kThreads);
  if (split) {
    const double rs = split_rho_scale(c->precision);
    if (smem > 48 * 1024)
      LRT_CUDA(cudaFuncSetAttribute(s0_project<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    s0_project<true><<<(unsigned)blocks, kThreads, smem, s>>>(
        rho, c->rho_ld, c->rho_gpad, N, u, v, pw, nullptr, nullptr, c->np, c->etas[j],
        pref / (rs * rs * (double)sB), out);
  } else {
    if (smem > 48 * 1024)
      LRT_CUDA(cudaFuncSetAttribute(s0_project<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    s0_project<false><<<(unsigned)blocks, kThreads, smem, s>>>(
        c->dw.rho, c->rho_ld, 0, N, u, v, nullptr, c->dw.delta, c->dw.df, c->np, c->etas[j], pref,
        out);
  }
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  (void)rho;
  return LRT_OK;
}

// d s/d theta of q at w = 0 (host ds[10], complex pairs), given on the device: u and v at w = 0,
// dK [3][N], FP64 Delta, df, d df/dT per pair, and this q's pair densities in dw.rho.
lrt_status launch_s0_tangents(const lrt_ctx* c, const QData& q, const double2* u, const double2* v,
                              const double* d_dK, const double* delta, const double* df,
                              const double* ddf, double* ds_host, cudaStream_t s) {
  const int N = q.nG;
  const size_t smem = ((size_t)N * ZCH + 6 * (size_t)N) * sizeof(double2);
  if (smem > 227 * 1024) {
    set_error("adjoint of S(q,0): N_G too large for the shared-memory tile");
    return LRT_EUNSUPPORTED;
  }
  double2* vec = c->dw.zf + 3 * (size_t)N;   // [4][N]
  double2* sc = vec + 4 * (size_t)N;         // [2]
  double2* y = sc + 2;                       // [N]
  double2* z = y + N;                        // [N]
  double2* ds = z + N;                       // [5]
  LRT_CUDA(cudaMemsetAsync(vec, 0, (4 * (size_t)N + 2) * sizeof(double2), s));
  int dev = 0, nsm = 0;
  LRT_CUDA(cudaGetDevice(&dev));
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  long long nb = std::max<long long>(1, std::min<long long>(2LL * nsm, (c->np + ZCH - 1) / ZCH));
  long long per = (c->np + nb - 1) / nb;
  per = (per + ZCH - 1) / ZCH * ZCH;
  nb = (c->np + per - 1) / per;
  const bool split = c->precision != LRT_PREC_FP64;
  const double rs = split ? (double)split_rho_scale(c->precision) : 1.0;
  const double scale = 2.0 / (c->nk * c->volume) / (rs * rs);
  if (split) {
    LRT_CUDA(cudaFuncSetAttribute(zf_vector_project<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    zf_vector_project<float2><<<(unsigned)nb, kThreads, smem, s>>>(
        (const float2*)c->dw.rho, c->rho_ld, c->rho_gpad, N, u, v, delta, df, ddf, c->np, per,
        c->eta, scale, vec, sc);
  } else {
    LRT_CUDA(cudaFuncSetAttribute(zf_vector_project<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    zf_vector_project<double2><<<(unsigned)nb, kThreads, smem, s>>>(
        (const double2*)c->dw.rho, c->rho_ld, 0, N, u, v, delta, df, ddf, c->np, per, c->eta,
        scale, vec, sc);
  }
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  // y = M^{-1} b_eta,  z = M^{-T} (K a_eta)
  LRT_TRY(launch_lu_two_solves(c, q, c->hcol, vec + 3 * (size_t)N, vec + N, q.Kdev, y, z, nullptr, s));
  zf_combine<<<1, kThreads, 0, s>>>(q.chi0 + (size_t)c->hcol * N * N, q.Kdev, d_dK,
                                    q.chi + (size_t)c->hcol * N, u, vec, sc, y, z, N, ds);
  count_launch(c);
  LRT_CUDA(cudaGetLastError());
  LRT_CUDA(cudaMemcpyAsync(ds_host, ds, 5 * sizeof(double2), cudaMemcpyDeviceToHost, s));
  LRT_CUDA(cudaStreamSynchronize(s));
  return LRT_OK;
}

}  // namespace lrt
