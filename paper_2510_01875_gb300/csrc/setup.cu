// Setup (not part of the timed response path): k meshes, plane-wave bases, response G-sets,
// the empty-core Hamiltonian H_GG'(k) = |k+G|^2/2 delta_GG' + V(G-G') assembled on the GPU
// and diagonalised by cuSOLVER, the kept eigenvectors refined by one first-order step in the
// solver's eigenbasis, Fermi-Dirac occupations with mu by bisection, and the Dyson kernel
// K_GG = 4 pi/|q+G|^2 + f_xc.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <thread>

#include "lrt_internal.h"

namespace lrt {

namespace {

struct V3 {
  double x, y, z;
};

V3 gvec(const lrt_ctx* c, int h, int k, int l) {
  return {h * c->recip[0][0] + k * c->recip[1][0] + l * c->recip[2][0],
          h * c->recip[0][1] + k * c->recip[1][1] + l * c->recip[2][1],
          h * c->recip[0][2] + k * c->recip[1][2] + l * c->recip[2][2]};
}

double norm3(const double* v) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

// Integer box containing every G with |center + G| <= radius: |m_i| <= (radius + |center|)
// |a_i| / (2 pi), plus one.
void miller_box(const lrt_ctx* c, const double* center, double radius, int lim[3]) {
  double reach = radius + norm3(center);
  for (int i = 0; i < 3; ++i)
    lim[i] = (int)std::ceil(reach * norm3(c->lattice[i]) / (2.0 * M_PI)) + 1;
}

// Basis {G : |k+G|^2 <= 2 ecut + tol} in lexicographic (h,k,l) order.
void sphere(const lrt_ctx* c, const double* k, std::vector<int32_t>& out) {
  out.clear();
  int lim[3];
  double zero[3] = {0, 0, 0};
  const double* ctr = (c->basis == LRT_BASIS_FIXED) ? zero : k;
  miller_box(c, ctr, std::sqrt(2.0 * c->ecut), lim);
  for (int h = -lim[0]; h <= lim[0]; ++h)
    for (int kk = -lim[1]; kk <= lim[1]; ++kk)
      for (int l = -lim[2]; l <= lim[2]; ++l) {
        V3 g = gvec(c, h, kk, l);
        double x = ctr[0] + g.x, y = ctr[1] + g.y, z = ctr[2] + g.z;
        if (x * x + y * y + z * z <= 2.0 * c->ecut + kBasisTol) {
          out.push_back(h);
          out.push_back(kk);
          out.push_back(l);
        }
      }
}

// Shell labels of values v: ascending order, a new shell whenever a value exceeds the first
// member of the current shell by more than kShellTol.
std::vector<int> shell_labels(const std::vector<double>& v) {
  std::vector<int> order(v.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return v[a] < v[b]; });
  std::vector<int> lab(v.size());
  int cur = -1;
  double start = 0.0;
  for (int idx : order) {
    if (cur < 0 || v[idx] - start > kShellTol) {
      ++cur;
      start = v[idx];
    }
    lab[idx] = cur;
  }
  return lab;
}

lrt_status response_gset(const lrt_ctx* c, const double* q, int nG, std::vector<int32_t>& out) {
  double radius = 1.0;
  std::vector<int32_t> cand;
  std::vector<double> d2;
  for (int iter = 0; iter < 60; ++iter) {
    int lim[3];
    miller_box(c, q, radius, lim);
    cand.clear();
    d2.clear();
    int well_inside = 0;
    for (int h = -lim[0]; h <= lim[0]; ++h)
      for (int k = -lim[1]; k <= lim[1]; ++k)
        for (int l = -lim[2]; l <= lim[2]; ++l) {
          V3 g = gvec(c, h, k, l);
          double x = q[0] + g.x, y = q[1] + g.y, z = q[2] + g.z;
          double v = x * x + y * y + z * z;
          if (v <= radius * radius) {
            cand.push_back(h);
            cand.push_back(k);
            cand.push_back(l);
            d2.push_back(v);
            if (v <= radius * radius - 1e-6) ++well_inside;
          }
        }
    if (well_inside >= nG) break;
    radius *= 1.5;
  }
  size_t n = d2.size();
  std::vector<double> g2(n);
  for (size_t i = 0; i < n; ++i) {
    V3 g = gvec(c, cand[3 * i], cand[3 * i + 1], cand[3 * i + 2]);
    g2[i] = g.x * g.x + g.y * g.y + g.z * g.z;
  }
  std::vector<int> s1 = shell_labels(d2), s2 = shell_labels(g2);
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    if (s1[a] != s1[b]) return s1[a] < s1[b];
    if (s2[a] != s2[b]) return s2[a] < s2[b];
    for (int j = 0; j < 3; ++j)
      if (cand[3 * a + j] != cand[3 * b + j]) return cand[3 * a + j] < cand[3 * b + j];
    return false;
  });
  if ((int)n < nG) {
    set_error("response G-set search failed");
    return LRT_EINVAL;
  }
  int zero = -1;
  for (int i = 0; i < nG; ++i) {
    int a = idx[i];
    if (cand[3 * a] == 0 && cand[3 * a + 1] == 0 && cand[3 * a + 2] == 0) zero = i;
  }
  if (zero < 0) {
    set_error("G = 0 is not among the nG vectors of smallest |q+G|");
    return LRT_EINVAL;
  }
  out.clear();
  out.push_back(0);
  out.push_back(0);
  out.push_back(0);
  for (int i = 0; i < nG; ++i) {
    if (i == zero) continue;
    int a = idx[i];
    out.push_back(cand[3 * a]);
    out.push_back(cand[3 * a + 1]);
    out.push_back(cand[3 * a + 2]);
  }
  return LRT_OK;
}

// Perdew-Wang 1992 unpolarised correlation energy per electron and its first two r_s
// derivatives: eps_c = -2A(1 + a1 r) L, L = ln(1 + 1/Q), Q = 2A(b1 r^1/2 + b2 r + b3 r^3/2
// + b4 r^2).  With D = Q(Q+1): eps' = -2A a1 L + 2A(1 + a1 r) Q'/D and
// eps'' = 4A a1 Q'/D + 2A(1 + a1 r)(Q''/D - Q'^2 (2Q + 1)/D^2).
void pw92(double r, double* e0, double* e1, double* e2) {
  const double A = 0.031091, a1 = 0.21370;
  const double b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
  double s = std::sqrt(r);
  double Q = 2.0 * A * (b1 * s + b2 * r + b3 * r * s + b4 * r * r);
  double Qp = 2.0 * A * (0.5 * b1 / s + b2 + 1.5 * b3 * s + 2.0 * b4 * r);
  double Qpp = 2.0 * A * (-0.25 * b1 / (r * s) + 0.75 * b3 / s + 2.0 * b4);
  double D = Q * (Q + 1.0);
  double L = std::log1p(1.0 / Q);
  double pre = 2.0 * A * (1.0 + a1 * r);
  *e0 = -pre * L;
  *e1 = -2.0 * A * a1 * L + pre * Qp / D;
  *e2 = 4.0 * A * a1 * Qp / D + pre * (Qpp / D - Qp * Qp * (2.0 * Q + 1.0) / (D * D));
}

}  // namespace

// f_xc = d^2(n eps_xc)/dn^2: exchange -pi/k_F^2; correlation (r^2 eps'' - 2 r eps')/(9 n).
double fxc_alda(double n) {
  double kf = std::cbrt(3.0 * M_PI * M_PI * n);
  double rs = std::cbrt(3.0 / (4.0 * M_PI * n));
  double e0, e1, e2;
  pw92(rs, &e0, &e1, &e2);
  return -M_PI / (kf * kf) + (rs * rs * e2 - 2.0 * rs * e1) / (9.0 * n);
}

double fxc_model(double qg, double n, double A, double B, double C) {
  return A * fxc_alda(n) * (1.0 + B * qg * qg) * std::exp(-C * qg * qg);
}

void kernel_diag(const lrt_ctx* c, QData& Q) {
  Q.K.resize(Q.nG);
  for (int g = 0; g < Q.nG; ++g) {
    const double qg2 = Q.qg2[g];
    double Kv = 4.0 * M_PI / qg2;
    if (c->kernel.kind == LRT_KERNEL_RPA_ALDA) Kv += c->fxc;
    if (c->kernel.kind == LRT_KERNEL_FXC_MODEL)
      Kv += fxc_model(std::sqrt(qg2), c->density, c->kernel.A, c->kernel.B, c->kernel.C);
    Q.K[g] = Kv;
  }
}

lrt_status build_geometry(lrt_ctx* c, const int* nG) {
  // reciprocal vectors b_j = 2 pi (a_k x a_l) / Omega
  const double(*a)[3] = c->lattice;
  double cr[3][3];
  for (int j = 0; j < 3; ++j) {
    const double* u = a[(j + 1) % 3];
    const double* v = a[(j + 2) % 3];
    cr[j][0] = u[1] * v[2] - u[2] * v[1];
    cr[j][1] = u[2] * v[0] - u[0] * v[2];
    cr[j][2] = u[0] * v[1] - u[1] * v[0];
  }
  double det = a[0][0] * cr[0][0] + a[0][1] * cr[0][1] + a[0][2] * cr[0][2];
  if (std::fabs(det) < 1e-12) {
    set_error("singular lattice");
    return LRT_EINVAL;
  }
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i) c->recip[j][i] = 2.0 * M_PI * cr[j][i] / det;
  c->volume = std::fabs(det);
  c->nelec = c->Z * c->natoms;
  c->density = c->nelec / c->volume;
  c->fxc = fxc_alda(c->density);

  c->qd.resize(c->nq);
  c->nGmax = 0;
  c->npw = 0;
  std::vector<std::vector<int32_t>> bases;
  for (int iq = 0; iq < c->nq; ++iq) {
    QData& Q = c->qd[iq];
    const double* qv = &c->q[3 * iq];
    // q must not be a reciprocal-lattice vector
    double red[3];
    for (int j = 0; j < 3; ++j)
      red[j] = (qv[0] * a[j][0] + qv[1] * a[j][1] + qv[2] * a[j][2]) / (2.0 * M_PI);
    if (std::fabs(red[0] - std::round(red[0])) < 1e-9 &&
        std::fabs(red[1] - std::round(red[1])) < 1e-9 &&
        std::fabs(red[2] - std::round(red[2])) < 1e-9) {
      set_error("q is a reciprocal-lattice vector");
      return LRT_EINVAL;
    }
    Q.nG = nG[iq];
    LRT_TRY(response_gset(c, qv, Q.nG, Q.gset));
    c->nGmax = std::max(c->nGmax, Q.nG);
    Q.qg2.resize(Q.nG);
    for (int g = 0; g < Q.nG; ++g) {
      V3 G = gvec(c, Q.gset[3 * g], Q.gset[3 * g + 1], Q.gset[3 * g + 2]);
      double x = qv[0] + G.x, y = qv[1] + G.y, z = qv[2] + G.z;
      Q.qg2[g] = x * x + y * y + z * z;
    }
    kernel_diag(c, Q);
    // meshes: k in M (+ shift), k+q = k + q
    double shift[3] = {0, 0, 0};
    if (c->kscheme == LRT_K_TR_SYMMETRIC)
      for (int j = 0; j < 3; ++j) shift[j] = -0.5 * qv[j];
    Q.kpts.resize(2 * c->nk * 3);
    int ik = 0;
    for (int i = 0; i < c->kn[0]; ++i)
      for (int j = 0; j < c->kn[1]; ++j)
        for (int l = 0; l < c->kn[2]; ++l, ++ik) {
          double fi = (double)i / c->kn[0], fj = (double)j / c->kn[1], fl = (double)l / c->kn[2];
          for (int x = 0; x < 3; ++x) {
            double kx = fi * c->recip[0][x] + fj * c->recip[1][x] + fl * c->recip[2][x] + shift[x];
            Q.kpts[3 * ik + x] = kx;
            Q.kpts[3 * (c->nk + ik) + x] = kx + qv[x];
          }
        }
    for (int s = 0; s < 2 * c->nk; ++s) {
      std::vector<int32_t> b;
      sphere(c, &Q.kpts[3 * s], b);
      c->npw = std::max(c->npw, (int)(b.size() / 3));
      if ((int)(b.size() / 3) < c->nb) {
        set_error("nbands exceeds the number of plane waves at a k point");
        return LRT_EINVAL;
      }
      bases.push_back(std::move(b));
    }
  }
  // padded Miller lists and gather tables (index of G1 + G in the k+q basis)
  int npw = c->npw;
  size_t bi = 0;
  for (int iq = 0; iq < c->nq; ++iq) {
    QData& Q = c->qd[iq];
    Q.miller.assign((size_t)2 * c->nk * npw * 3, INT32_MIN);
    Q.npw_k.resize(2 * c->nk);
    for (int s = 0; s < 2 * c->nk; ++s, ++bi) {
      const std::vector<int32_t>& b = bases[bi];
      Q.npw_k[s] = (int32_t)(b.size() / 3);
      std::copy(b.begin(), b.end(), Q.miller.begin() + (size_t)s * npw * 3);
    }
  }
  return LRT_OK;
}

namespace {

// Gather table for one q: gather[k][g][j] = index in the k+q basis of G1_j + G_g, or -1.
void build_gather(const lrt_ctx* c, const QData& Q, std::vector<int32_t>& tab) {
  int nk = c->nk, npw = c->npw, nG = Q.nG;
  tab.assign((size_t)nk * nG * npw, -1);
  auto work = [&](int k0, int k1) {
    std::vector<int32_t> lut;
    for (int k = k0; k < k1; ++k) {
      const int32_t* mk = &Q.miller[(size_t)k * npw * 3];
      const int32_t* mq = &Q.miller[(size_t)(nk + k) * npw * 3];
      int nq = Q.npw_k[nk + k], nkk = Q.npw_k[k];
      int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
      for (int j = 0; j < nq; ++j)
        for (int x = 0; x < 3; ++x) {
          lo[x] = std::min(lo[x], mq[3 * j + x]);
          hi[x] = std::max(hi[x], mq[3 * j + x]);
        }
      int ext[3] = {hi[0] - lo[0] + 1, hi[1] - lo[1] + 1, hi[2] - lo[2] + 1};
      lut.assign((size_t)ext[0] * ext[1] * ext[2], -1);
      for (int j = 0; j < nq; ++j)
        lut[((size_t)(mq[3 * j] - lo[0]) * ext[1] + (mq[3 * j + 1] - lo[1])) * ext[2] +
            (mq[3 * j + 2] - lo[2])] = j;
      for (int g = 0; g < nG; ++g) {
        int32_t* row = &tab[((size_t)k * nG + g) * npw];
        for (int j = 0; j < nkk; ++j) {
          int t0 = mk[3 * j] + Q.gset[3 * g] - lo[0];
          int t1 = mk[3 * j + 1] + Q.gset[3 * g + 1] - lo[1];
          int t2 = mk[3 * j + 2] + Q.gset[3 * g + 2] - lo[2];
          if (t0 < 0 || t1 < 0 || t2 < 0 || t0 >= ext[0] || t1 >= ext[1] || t2 >= ext[2]) continue;
          row[j] = lut[((size_t)t0 * ext[1] + t1) * ext[2] + t2];
        }
      }
    }
  };
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  int per = (nk + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    int k0 = t * per, k1 = std::min(nk, k0 + per);
    if (k0 < k1) th.emplace_back(work, k0, k1);
  }
  for (auto& t : th) t.join();
}

// H assembly, column-major per matrix (A[i + j*npw]):
// A_ij = |k+G_i|^2/2 delta_ij + V(G_i - G_j); padding rows/cols: kPadDiag on the diagonal.
__global__ void assemble_h(double2* __restrict__ A, const int32_t* __restrict__ miller,
                           const int32_t* __restrict__ npw_k, const double* __restrict__ kpts,
                           int npw, int nmat, const double* __restrict__ pos, int natoms,
                           double3 b0, double3 b1, double3 b2, double Z, double rc, double vol,
                           int zero_potential) {
  int64_t total = (int64_t)nmat * npw * npw;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t % npw);
    int j = (int)((t / npw) % npw);
    int m = (int)(t / ((int64_t)npw * npw));
    int n = npw_k[m];
    double2 v = make_double2(0.0, 0.0);
    if (i >= n || j >= n) {
      if (i == j) v.x = kPadDiag;
    } else {
      const int32_t* mi = miller + ((size_t)m * npw + i) * 3;
      const int32_t* mj = miller + ((size_t)m * npw + j) * 3;
      if (i == j) {
        double kx = kpts[3 * m] + mi[0] * b0.x + mi[1] * b1.x + mi[2] * b2.x;
        double ky = kpts[3 * m + 1] + mi[0] * b0.y + mi[1] * b1.y + mi[2] * b2.y;
        double kz = kpts[3 * m + 2] + mi[0] * b0.z + mi[1] * b1.z + mi[2] * b2.z;
        v.x = 0.5 * (kx * kx + ky * ky + kz * kz);
      } else if (!zero_potential) {
        int h = mi[0] - mj[0], k = mi[1] - mj[1], l = mi[2] - mj[2];
        double gx = h * b0.x + k * b1.x + l * b2.x;
        double gy = h * b0.y + k * b1.y + l * b2.y;
        double gz = h * b0.z + k * b1.z + l * b2.z;
        double g2 = gx * gx + gy * gy + gz * gz;
        double g = sqrt(g2);
        double ff = -(4.0 * M_PI * Z / (vol * g2)) * cos(g * rc);
        double sr = 0.0, si = 0.0;
        for (int a = 0; a < natoms; ++a) {
          double ph = gx * pos[3 * a] + gy * pos[3 * a + 1] + gz * pos[3 * a + 2];
          double s, c;
          sincos(ph, &s, &c);
          sr += c;
          si -= s;
        }
        v.x = ff * sr;
        v.y = ff * si;
      }
    }
    A[((size_t)m * npw + j) * npw + i] = v;
  }
}

// eps[m][n] = W[m][n]; coeff[m][n][g] = A[m][g + n*npw] (g < npw_k, else 0), n < nb.
__global__ void extract_eigen(const double2* __restrict__ A, const double* __restrict__ W,
                              const int32_t* __restrict__ npw_k, int npw, int nb, int nmat,
                              double* __restrict__ eps, double2* __restrict__ coeff) {
  int64_t total = (int64_t)nmat * nb * npw;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int g = (int)(t % npw);
    int n = (int)((t / npw) % nb);
    int m = (int)(t / ((int64_t)npw * nb));
    double2 v = A[((size_t)m * npw + n) * npw + g];
    if (g >= npw_k[m]) v = make_double2(0.0, 0.0);
    coeff[t] = v;
    if (g == 0) eps[(size_t)m * nb + n] = W[(size_t)m * npw + n];
  }
}

// First-order correction coefficients of the kept eigenvectors from E = V^H H V_kept
// ([npw][nb] column-major per matrix, W the solver's ascending eigenvalues):
//   C_ij = E_ij / (eps_j - eps_i) for i != j, 0 on the diagonal and for pairs closer than
//   kDegenTol or with |E_ij| not small against the gap (near-degenerate pairs: any rotation
//   inside them is an eigenbasis to this accuracy).
__global__ void refine_coeffs(double2* __restrict__ E, const double* __restrict__ W, int npw, int nb,
                              int nmat) {
  int64_t total = (int64_t)nmat * nb * npw;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % npw);
    const int j = (int)((t / npw) % nb);
    const int m = (int)(t / ((int64_t)npw * nb));
    const double gap = W[(size_t)m * npw + j] - W[(size_t)m * npw + i];
    const double2 e = E[t];
    double2 c = make_double2(0.0, 0.0);
    if (i != j && fabs(gap) > kDegenTol && sqrt(e.x * e.x + e.y * e.y) < 1e-3 * fabs(gap))
      c = make_double2(e.x / gap, e.y / gap);
    E[t] = c;
  }
}

// W[m][j] = Re v_j^H (H v_j) for the first nb columns (Rayleigh quotients of the refined
// vectors; HV = H V_kept [npw][nb] per matrix).  One warp per (matrix, column).
__global__ void rayleigh_quotients(const double2* __restrict__ V, const double2* __restrict__ HV,
                                   int npw, int nb, int nmat, double* __restrict__ W) {
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (long long)nmat * nb) return;
  const int m = (int)(warp / nb), j = (int)(warp % nb);
  const double2* v = V + (size_t)m * npw * npw + (size_t)j * npw;
  const double2* h = HV + (size_t)m * npw * nb + (size_t)j * npw;
  double acc = 0.0;
  for (int g = lane; g < npw; g += 32) acc += v[g].x * h[g].x + v[g].y * h[g].y;
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) W[(size_t)m * npw + j] = acc;
}

// S <- 3/2 I - S/2 per [nb][nb] matrix (one Lowdin step: (V^H V)^{-1/2} to second order).
__global__ void lowdin_factor(double2* __restrict__ S, int nb, int nmat) {
  int64_t total = (int64_t)nmat * nb * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % nb), j = (int)((t / nb) % nb);
    double2 v = S[t];
    v = make_double2(-0.5 * v.x, -0.5 * v.y);
    if (i == j) v.x += 1.5;
    S[t] = v;
  }
}

struct Solver {
  cusolverDnHandle_t h = nullptr;
  cusolverDnParams_t p = nullptr;
  cublasHandle_t b = nullptr;
  ~Solver() {
    if (p) cusolverDnDestroyParams(p);
    if (h) cusolverDnDestroy(h);
    if (b) cublasDestroy(b);
  }
};

#define LRT_BLAS(call)                                                     \
  do {                                                                     \
    cublasStatus_t st_ = (call);                                           \
    if (st_ != CUBLAS_STATUS_SUCCESS) {                                    \
      set_error(std::string(#call) + " failed: " + std::to_string(st_));   \
      return LRT_ECUDA;                                                    \
    }                                                                      \
  } while (0)

// One refinement step of the nb kept eigenvectors of nm matrices: V (npw x npw per matrix,
// column-major, the solver's full eigenbasis) and W (its eigenvalues); Hm holds the same
// Hamiltonians; T1, T2 are [npw][nb] and Sm [nb][nb] per matrix.  The batched solver's vectors
// carry residuals ||H v - eps v|| up to ~1e-9 Ha; the correction
//   v_j <- v_j + sum_i v_i C_ij,  C = refine_coeffs(V^H H V_kept)
// removes them to first order (the residual then falls quadratically), and one Lowdin step
// V <- V (3/2 I - (V^H V)/2) restores orthonormality to second order.  The corrected vectors
// replace the first nb columns of V, and their Rayleigh quotients replace the first nb
// eigenvalues in W (the solver's eigenvalues carried errors up to ~1e-11 Ha, larger than the
// refined vectors' residuals).
lrt_status refine_kept(const Solver& sv, double2* V, double* W, const double2* Hm, double2* T1,
                       double2* T2, double2* Sm, int npw, int nb, int nm) {
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  const long long sM = (long long)npw * npw, sT = (long long)npw * nb, sS = (long long)nb * nb;
  auto Z = [](const double2* p) { return reinterpret_cast<const cuDoubleComplex*>(p); };
  auto Zm = [](double2* p) { return reinterpret_cast<cuDoubleComplex*>(p); };
  // T1 = H V_kept;  T2 = V^H T1
  LRT_BLAS(cublasZgemmStridedBatched(sv.b, CUBLAS_OP_N, CUBLAS_OP_N, npw, nb, npw, &one, Z(Hm), npw,
                                     sM, Z(V), npw, sM, &zero, Zm(T1), npw, sT, nm));
  LRT_BLAS(cublasZgemmStridedBatched(sv.b, CUBLAS_OP_C, CUBLAS_OP_N, npw, nb, npw, &one, Z(V), npw,
                                     sM, Z(T1), npw, sT, &zero, Zm(T2), npw, sT, nm));
  refine_coeffs<<<1216, 256>>>(T2, W, npw, nb, nm);
  LRT_CUDA(cudaGetLastError());
  // T1 = V_kept + V C
  LRT_CUDA(cudaMemcpy2D(T1, sT * sizeof(double2), V, sM * sizeof(double2), sT * sizeof(double2), nm,
                        cudaMemcpyDeviceToDevice));
  LRT_BLAS(cublasZgemmStridedBatched(sv.b, CUBLAS_OP_N, CUBLAS_OP_N, npw, nb, npw, &one, Z(V), npw,
                                     sM, Z(T2), npw, sT, &one, Zm(T1), npw, sT, nm));
  // S = T1^H T1;  V_kept = T1 (3/2 I - S/2)
  LRT_BLAS(cublasZgemmStridedBatched(sv.b, CUBLAS_OP_C, CUBLAS_OP_N, nb, nb, npw, &one, Z(T1), npw,
                                     sT, Z(T1), npw, sT, &zero, Zm(Sm), nb, sS, nm));
  lowdin_factor<<<1216, 256>>>(Sm, nb, nm);
  LRT_CUDA(cudaGetLastError());
  LRT_BLAS(cublasZgemmStridedBatched(sv.b, CUBLAS_OP_N, CUBLAS_OP_N, npw, nb, nb, &one, Z(T1), npw,
                                     sT, Z(Sm), nb, sS, &zero, Zm(V), npw, sM, nm));
  // eigenvalues: Rayleigh quotients of the refined vectors
  LRT_BLAS(cublasZgemmStridedBatched(sv.b, CUBLAS_OP_N, CUBLAS_OP_N, npw, nb, npw, &one, Z(Hm), npw,
                                     sM, Z(V), npw, sM, &zero, Zm(T1), npw, sT, nm));
  const long long warps = (long long)nm * nb;
  rayleigh_quotients<<<(unsigned)((warps * 32 + 255) / 256), 256>>>(V, T1, npw, nb, nm, W);
  LRT_CUDA(cudaGetLastError());
  return LRT_OK;
}

#define LRT_SOLVER(call)                                                   \
  do {                                                                     \
    cusolverStatus_t st_ = (call);                                         \
    if (st_ != CUSOLVER_STATUS_SUCCESS) {                                  \
      set_error(std::string(#call) + " failed: " + std::to_string(st_));   \
      return LRT_ECUDA;                                                    \
    }                                                                      \
  } while (0)

double fermi(double e, double mu, double T) {
  double x = (e - mu) / T;
  if (x > 0) {
    double ex = std::exp(-x);
    return ex / (1.0 + ex);
  }
  return 1.0 / (1.0 + std::exp(x));
}

}  // namespace

// Band weights of one k point from its nfull ascending eigenvalues: 1 for the lowest nbands,
// 0 above; a multiplet within kDegenTol of the last kept band that the cut splits (j of its
// m members kept) gives each member j/m, which makes the kept projector gauge-invariant.
// Returns the number of bands with nonzero weight, or -1 if the multiplet reaches the last
// computed band (so that members above it could be missing) and `complete` is false.
int band_weights(const double* e, int nfull, int nbands, double* w, bool complete = false) {
  for (int n = 0; n < nfull; ++n) w[n] = n < nbands ? 1.0 : 0.0;
  const double last = e[nbands - 1];
  int lo = nbands - 1, hi = nbands - 1;
  for (int n = 0; n < nfull; ++n)
    if (std::fabs(e[n] - last) <= kDegenTol) {
      lo = std::min(lo, n);
      hi = std::max(hi, n);
    }
  int m = hi - lo + 1, j = nbands - lo;
  if (m == j) return nbands;
  if (hi >= nfull - 1 && !complete) return -1;
  for (int n = lo; n <= hi; ++n) w[n] = (double)j / m;
  return hi + 1;
}

// mu by 200 halvings of [min eps - 60 T, max eps + 60 T] so that (2/N_k) sum w f = N_e over
// the k mesh of q (wgt: band weights of both meshes); f [2 nk nb] on both meshes.
lrt_status fermi_occupations(const lrt_ctx* c, const double* eps_host, const double* wg,
                             double* f, double* mu_out) {
  int nk = c->nk, nb = c->nb;
  size_t half = (size_t)nk * nb;
  double cap = 0.0;
  for (size_t i = 0; i < half; ++i) cap += wg[i];
  if (2.0 * cap / nk < c->nelec) {
    set_error("not enough bands to hold the electrons");
    return LRT_EINVAL;
  }
  double lo = eps_host[0], hi = eps_host[0];
  for (size_t i = 0; i < half; ++i) {
    lo = std::min(lo, eps_host[i]);
    hi = std::max(hi, eps_host[i]);
  }
  lo -= 60.0 * c->T;
  hi += 60.0 * c->T;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double s = 0.0;
    for (size_t i = 0; i < half; ++i) s += wg[i] * fermi(eps_host[i], mid, c->T);
    if (2.0 * s / nk < c->nelec)
      lo = mid;
    else
      hi = mid;
    if (hi - lo <= 0.0) break;
  }
  const double mu = 0.5 * (lo + hi);
  *mu_out = mu;
  for (size_t i = 0; i < 2 * half; ++i) f[i] = fermi(eps_host[i], mu, c->T);
  return LRT_OK;
}

// Fermi-Dirac occupations of q from host eigenvalues and the q's band weights, uploaded.
lrt_status set_occupations_fd(lrt_ctx* c, int iq, const double* eps_host) {
  QData& Q = c->qd[iq];
  std::vector<double> f((size_t)2 * c->nk * c->nb);
  LRT_TRY(fermi_occupations(c, eps_host, Q.wgt_h.data(), f.data(), &Q.mu));
  LRT_CUDA(cudaMemcpy(Q.occ, f.data(), f.size() * sizeof(double), cudaMemcpyHostToDevice));
  return LRT_OK;
}

lrt_status solve_ground_states(lrt_ctx* c, const double* occupations) {
  int nk = c->nk, npw = c->npw;
  // eigenpairs kept per k before the band weights are known: nbands plus room for a
  // multiplet split by the cut
  int npw_min = npw;
  for (auto& Q : c->qd)
    for (int v : Q.npw_k) npw_min = std::min(npw_min, v);
  const int nb = std::min(npw_min, c->nbands + kExtraBands);
  size_t per_mat = (size_t)npw * npw * sizeof(double2);
  int total = 2 * nk * c->nq;
  // batch of matrices per eigensolver call (about 3 GB of matrices)
  int batch = (int)std::max<size_t>(1, std::min<size_t>(total, (size_t)3e9 / per_mat));
  for (int iq = 0; iq < c->nq; ++iq) {
    QData& Q = c->qd[iq];
    LRT_CUDA(cudaMalloc(&Q.eps, 2 * (size_t)nk * nb * sizeof(double)));
    LRT_CUDA(cudaMalloc(&Q.occ, 2 * (size_t)nk * nb * sizeof(double)));
    LRT_CUDA(cudaMalloc(&Q.coeff, 2 * (size_t)nk * nb * npw * sizeof(double2)));
    std::vector<int32_t> tab;
    build_gather(c, Q, tab);
    LRT_CUDA(cudaMalloc(&Q.gather, tab.size() * sizeof(int32_t)));
    LRT_CUDA(cudaMemcpy(Q.gather, tab.data(), tab.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  Solver sv;
  LRT_SOLVER(cusolverDnCreate(&sv.h));
  LRT_SOLVER(cusolverDnCreateParams(&sv.p));
  LRT_BLAS(cublasCreate(&sv.b));
  // standard FP64 arithmetic in the refinement products (no emulated or reduced-precision
  // algorithms): they must resolve residuals far below the solver's
  LRT_BLAS(cublasSetMathMode(sv.b, CUBLAS_PEDANTIC_MATH));
  double2* A = nullptr;
  double2 *Hm = nullptr, *T1 = nullptr, *T2 = nullptr, *Sm = nullptr;
  double* W = nullptr;
  int* info = nullptr;
  int32_t *d_miller = nullptr, *d_npw = nullptr;
  double *d_k = nullptr, *d_pos = nullptr;
  void* dwork = nullptr;
  std::vector<char> hwork;
  auto cleanup = [&]() {
    cudaFree(A);
    cudaFree(W);
    cudaFree(info);
    cudaFree(d_miller);
    cudaFree(d_npw);
    cudaFree(d_k);
    cudaFree(d_pos);
    cudaFree(dwork);
    cudaFree(Hm);
    cudaFree(T1);
    cudaFree(T2);
    cudaFree(Sm);
  };
  struct Guard {
    std::function<void()> f;
    ~Guard() { f(); }
  } guard{cleanup};
  LRT_CUDA(cudaMalloc(&A, per_mat * batch));
  LRT_CUDA(cudaMalloc(&Hm, per_mat * batch));
  LRT_CUDA(cudaMalloc(&T1, (size_t)npw * nb * batch * sizeof(double2)));
  LRT_CUDA(cudaMalloc(&T2, (size_t)npw * nb * batch * sizeof(double2)));
  LRT_CUDA(cudaMalloc(&Sm, (size_t)nb * nb * batch * sizeof(double2)));
  LRT_CUDA(cudaMalloc(&W, (size_t)npw * batch * sizeof(double)));
  LRT_CUDA(cudaMalloc(&info, batch * sizeof(int)));
  LRT_CUDA(cudaMalloc(&d_miller, (size_t)batch * npw * 3 * sizeof(int32_t)));
  LRT_CUDA(cudaMalloc(&d_npw, batch * sizeof(int32_t)));
  LRT_CUDA(cudaMalloc(&d_k, (size_t)batch * 3 * sizeof(double)));
  LRT_CUDA(cudaMalloc(&d_pos, std::max(1, c->natoms) * 3 * sizeof(double)));
  if (c->natoms)
    LRT_CUDA(cudaMemcpy(d_pos, c->positions.data(), c->natoms * 3 * sizeof(double),
                        cudaMemcpyHostToDevice));
  // batched solver if this cuSOLVER supports the size, else one matrix at a time
  size_t dws = 0, hws = 0;
  bool batched = cusolverDnXsyevBatched_bufferSize(
                     sv.h, sv.p, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, npw,
                     CUDA_C_64F, A, npw, CUDA_R_64F, W, CUDA_C_64F, &dws, &hws,
                     batch) == CUSOLVER_STATUS_SUCCESS;
  if (!batched) {
    LRT_SOLVER(cusolverDnXsyevd_bufferSize(sv.h, sv.p, CUSOLVER_EIG_MODE_VECTOR,
                                           CUBLAS_FILL_MODE_LOWER, npw, CUDA_C_64F, A, npw,
                                           CUDA_R_64F, W, CUDA_C_64F, &dws, &hws));
  }
  LRT_CUDA(cudaMalloc(&dwork, std::max<size_t>(dws, 16)));
  hwork.resize(std::max<size_t>(hws, 16));

  double3 b0 = make_double3(c->recip[0][0], c->recip[0][1], c->recip[0][2]);
  double3 b1 = make_double3(c->recip[1][0], c->recip[1][1], c->recip[1][2]);
  double3 b2 = make_double3(c->recip[2][0], c->recip[2][1], c->recip[2][2]);
  // enumerate (q, mesh point) in order and process in batches
  std::vector<int> info_h(batch);
  for (int start = 0; start < total; start += batch) {
    int nm = std::min(batch, total - start);
    std::vector<int32_t> hm((size_t)nm * npw * 3), hn(nm);
    std::vector<double> hk((size_t)nm * 3);
    for (int m = 0; m < nm; ++m) {
      int gidx = start + m;
      int iq = gidx / (2 * nk), s = gidx % (2 * nk);
      const QData& Q = c->qd[iq];
      std::copy(Q.miller.begin() + (size_t)s * npw * 3, Q.miller.begin() + (size_t)(s + 1) * npw * 3,
                hm.begin() + (size_t)m * npw * 3);
      hn[m] = Q.npw_k[s];
      for (int x = 0; x < 3; ++x) hk[3 * m + x] = Q.kpts[3 * s + x];
    }
    LRT_CUDA(cudaMemcpy(d_miller, hm.data(), hm.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    LRT_CUDA(cudaMemcpy(d_npw, hn.data(), nm * sizeof(int32_t), cudaMemcpyHostToDevice));
    LRT_CUDA(cudaMemcpy(d_k, hk.data(), hk.size() * sizeof(double), cudaMemcpyHostToDevice));
    assemble_h<<<1216, 256>>>(A, d_miller, d_npw, d_k, npw, nm, d_pos, c->natoms, b0, b1, b2, c->Z,
                              c->r_c, c->volume, c->potential == LRT_POT_ZERO);
    LRT_CUDA(cudaGetLastError());
    if (batched) {
      LRT_SOLVER(cusolverDnXsyevBatched(sv.h, sv.p, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                        npw, CUDA_C_64F, A, npw, CUDA_R_64F, W, CUDA_C_64F, dwork,
                                        dws, hwork.data(), hws, info, nm));
    } else {
      for (int m = 0; m < nm; ++m)
        LRT_SOLVER(cusolverDnXsyevd(sv.h, sv.p, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, npw,
                                    CUDA_C_64F, A + (size_t)m * npw * npw, npw, CUDA_R_64F,
                                    W + (size_t)m * npw, CUDA_C_64F, dwork, dws, hwork.data(), hws,
                                    info + m));
    }
    LRT_CUDA(cudaMemcpy(info_h.data(), info, nm * sizeof(int), cudaMemcpyDeviceToHost));
    for (int m = 0; m < nm; ++m)
      if (info_h[m] != 0) {
        set_error("eigensolver did not converge (info " + std::to_string(info_h[m]) + ")");
        return LRT_ECUDA;
      }
    // the solver overwrote A with the eigenvectors: H again, then refine the kept vectors
    assemble_h<<<1216, 256>>>(Hm, d_miller, d_npw, d_k, npw, nm, d_pos, c->natoms, b0, b1, b2, c->Z,
                              c->r_c, c->volume, c->potential == LRT_POT_ZERO);
    LRT_CUDA(cudaGetLastError());
    LRT_TRY(refine_kept(sv, A, W, Hm, T1, T2, Sm, npw, nb, nm));
    // scatter into the per-q arrays; a batch may straddle q boundaries
    for (int m0 = 0; m0 < nm;) {
      int gidx = start + m0;
      int iq = gidx / (2 * nk), s = gidx % (2 * nk);
      int run = std::min(nm - m0, 2 * nk - s);
      QData& Q = c->qd[iq];
      extract_eigen<<<1216, 256>>>(A + (size_t)m0 * npw * npw, W + (size_t)m0 * npw, d_npw + m0, npw,
                                   nb, run, Q.eps + (size_t)s * nb,
                                   Q.coeff + (size_t)s * nb * npw);
      LRT_CUDA(cudaGetLastError());
      m0 += run;
    }
  }
  LRT_CUDA(cudaDeviceSynchronize());
  // band weights and the number of bands carried (global over q)
  std::vector<std::vector<double>> eps_all(c->nq), w_all(c->nq);
  int nb_used = c->nbands;
  for (int iq = 0; iq < c->nq; ++iq) {
    eps_all[iq].resize((size_t)2 * nk * nb);
    w_all[iq].resize((size_t)2 * nk * nb);
    LRT_CUDA(cudaMemcpy(eps_all[iq].data(), c->qd[iq].eps, eps_all[iq].size() * sizeof(double),
                        cudaMemcpyDeviceToHost));
    for (int s = 0; s < 2 * nk; ++s) {
      double* w = &w_all[iq][(size_t)s * nb];
      if (occupations) {
        for (int n = 0; n < nb; ++n) w[n] = n < c->nbands ? 1.0 : 0.0;
        continue;
      }
      int used = band_weights(&eps_all[iq][(size_t)s * nb], nb, c->nbands, w);
      if (used < 0) {
        set_error("a degenerate multiplet at the band cut extends past the computed bands");
        return LRT_EINVAL;
      }
      nb_used = std::max(nb_used, used);
    }
  }
  // compact every q to nb_used bands
  c->nb = nb_used;
  for (int iq = 0; iq < c->nq; ++iq) {
    QData& Q = c->qd[iq];
    if (nb_used < nb) {
      double* e2 = nullptr;
      double2* c2 = nullptr;
      LRT_CUDA(cudaMalloc(&e2, (size_t)2 * nk * nb_used * sizeof(double)));
      LRT_CUDA(cudaMalloc(&c2, (size_t)2 * nk * nb_used * npw * sizeof(double2)));
      LRT_CUDA(cudaMemcpy2D(e2, nb_used * sizeof(double), Q.eps, nb * sizeof(double),
                            nb_used * sizeof(double), 2 * nk, cudaMemcpyDeviceToDevice));
      LRT_CUDA(cudaMemcpy2D(c2, (size_t)nb_used * npw * sizeof(double2), Q.coeff,
                            (size_t)nb * npw * sizeof(double2), (size_t)nb_used * npw * sizeof(double2),
                            2 * nk, cudaMemcpyDeviceToDevice));
      cudaFree(Q.eps);
      cudaFree(Q.coeff);
      Q.eps = e2;
      Q.coeff = c2;
      cudaFree(Q.occ);
      Q.occ = nullptr;
      LRT_CUDA(cudaMalloc(&Q.occ, (size_t)2 * nk * nb_used * sizeof(double)));
    }
    Q.wgt_h.resize((size_t)2 * nk * nb_used);
    std::vector<double> e((size_t)2 * nk * nb_used);
    for (int s = 0; s < 2 * nk; ++s)
      for (int n = 0; n < nb_used; ++n) {
        Q.wgt_h[(size_t)s * nb_used + n] = w_all[iq][(size_t)s * nb + n];
        e[(size_t)s * nb_used + n] = eps_all[iq][(size_t)s * nb + n];
      }
    LRT_CUDA(cudaMalloc(&Q.wgt, Q.wgt_h.size() * sizeof(double)));
    LRT_CUDA(cudaMemcpy(Q.wgt, Q.wgt_h.data(), Q.wgt_h.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (occupations) {
      // caller's f for the nominal bands, zero above
      Q.mu = NAN;
      std::vector<double> f((size_t)2 * nk * nb_used, 0.0);
      for (int s = 0; s < 2 * nk; ++s)
        for (int n = 0; n < c->nbands; ++n)
          f[(size_t)s * nb_used + n] = occupations[((size_t)iq * 2 * nk + s) * c->nbands + n];
      LRT_CUDA(cudaMemcpy(Q.occ, f.data(), f.size() * sizeof(double), cudaMemcpyHostToDevice));
    } else {
      LRT_TRY(set_occupations_fd(c, iq, e.data()));
    }
  }
  c->np = (int64_t)nk * c->nb * c->nb;
  c->rho_ld = (c->np + 31) / 32 * 32;
  c->rho_gpad = (c->precision == LRT_PREC_FP64) ? 0 : (c->nGmax + 7) / 8 * 8;
  return LRT_OK;
}

// Band weights of both meshes [2 nk nb] from eigenvalues supplied through the orbital hook.
lrt_status band_weights_all(const lrt_ctx* c, const double* eps_host, double* out) {
  const int nb = c->nb;
  for (int s = 0; s < 2 * c->nk; ++s) {
    // the context's nb already holds every member of a multiplet split at setup
    int used = band_weights(eps_host + (size_t)s * nb, nb, c->nbands, out + (size_t)s * nb, true);
    if (used < 0) {
      set_error("a degenerate multiplet at the band cut extends past the supplied bands");
      return LRT_EINVAL;
    }
  }
  return LRT_OK;
}

// Band weights recomputed from eigenvalues supplied through the orbital hook, uploaded.
lrt_status reset_band_weights(lrt_ctx* c, int iq, const double* eps_host) {
  QData& Q = c->qd[iq];
  LRT_TRY(band_weights_all(c, eps_host, Q.wgt_h.data()));
  LRT_CUDA(cudaMemcpy(Q.wgt, Q.wgt_h.data(), Q.wgt_h.size() * sizeof(double), cudaMemcpyHostToDevice));
  return LRT_OK;
}

}  // namespace lrt
