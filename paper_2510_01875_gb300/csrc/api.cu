// C ABI entry points of liblrtddft (declared in include/lrtddft.h): validation, context
// lifetime, the order of the response steps and host/device transfers.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "lrt_internal.h"

namespace lrt {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error() { return g_last_error.c_str(); }

namespace {

lrt_status bad(const char* msg) {
  set_error(msg);
  return LRT_EINVAL;
}

void free_events(lrt_ctx* c) {
  for (auto& e : c->ev_chi0) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto& e : c->ev_rho) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
}

void free_ctx(lrt_ctx* c) {
  if (!c) return;
  if (!c->host_only) free_events(c);
  if (c->host_only) {
    delete c;
    return;
  }
  cudaSetDevice(c->device);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  free_tc_state(c);
  free_kg_state(c);
  free_spectral_state(c);
  if (c->upload) {
    cudaStreamSynchronize(c->upload);
    cudaStreamDestroy(c->upload);
  }
  for (auto& q : c->qd) {
    cudaFree(q.up.coeff);
    cudaFree(q.up.eps);
    cudaFree(q.up.occ);
    cudaFree(q.up.wgt);
    cudaFreeHost(q.up.stage);
    if (q.up.ready) cudaEventDestroy(q.up.ready);
    if (q.up.free) cudaEventDestroy(q.up.free);
    free_split_plan(q.sp);
    cudaFree(q.Kdev);
    cudaFree(q.eps);
    cudaFree(q.occ);
    cudaFree(q.wgt);
    cudaFree(q.coeff);
    cudaFree(q.gather);
    cudaFree(q.chi0);
    cudaFree(q.chi);
  }
  cudaFree(c->dw.rho);
  cudaFree(c->dw.delta);
  cudaFree(c->dw.df);
  cudaFree(c->dw.freqs);
  cudaFree(c->dw.omega);
  cudaFree(c->dw.S);
  cudaFree(c->dw.chi00);
  cudaFree(c->dw.status);
  cudaFree(c->dw.scratch);
  cudaFree(c->dw.pd_work);
  cudaFree(c->dw.zt_part);
  cudaFree(c->dw.dyson_ws);
  cudaFree(c->dw.s0);
  cudaFree(c->dw.zf);
  cudaFree(c->dw.zf_ws);
  cudaFree(c->dw.eta_ref);
  delete c;
}

}  // namespace

// The device status word after the work so far: a timed-out wait (bit 2) first, then a zero
// Dyson pivot (bit 1).
lrt_status check_status_word(const lrt_ctx* c) {
  int st = 0;
  LRT_CUDA(cudaMemcpy(&st, c->dw.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st & 2) {
    set_error("a bounded device wait ran out");
    return LRT_ETIMEOUT;
  }
  if (st & 1) {
    set_error("zero pivot in a Dyson matrix");
    return LRT_ESINGULAR;
  }
  return LRT_OK;
}

lrt_status ensure_rho(lrt_ctx* c) {
  size_t elem = (c->precision == LRT_PREC_FP64) ? sizeof(double2) : sizeof(float2);
  size_t need = (size_t)(c->rho_gpad ? c->rho_gpad : c->nGmax) * c->rho_ld * elem;
  if (c->dw.rho_bytes >= need) return LRT_OK;
  cudaFree(c->dw.rho);
  c->dw.rho = nullptr;
  LRT_CUDA(cudaMalloc(&c->dw.rho, need));
  c->dw.rho_bytes = need;
  // padding (pairs past the last one, G rows past nG) is never written and must read as zero
  LRT_CUDA(cudaMemset(c->dw.rho, 0, need));
  LRT_CUDA(cudaDeviceSynchronize());
  return LRT_OK;
}

}  // namespace lrt

using namespace lrt;

extern "C" const char* lrtddft_status_string(lrt_status s) {
  switch (s) {
    case LRT_OK: return "ok";
    case LRT_EINVAL: return "invalid argument";
    case LRT_ENOMEM: return "out of memory";
    case LRT_ECUDA: return "CUDA error";
    case LRT_ESINGULAR: return "singular Dyson matrix";
    case LRT_ETIMEOUT: return "device wait timed out";
    case LRT_ESTATE: return "calls out of order";
    case LRT_EUNSUPPORTED: return "unsupported option";
  }
  return "unknown status";
}

extern "C" const char* lrtddft_last_error(void) { return lrt::last_error(); }

extern "C" lrt_status lrtddft_create(const lrt_cell* cell, const lrt_kmesh* kmesh, int nbands,
                                     double T, const double* occupations, int nq, const double* q,
                                     const int* nG, int nw, const double* omega, double eta,
                                     const lrt_kernel* kernel, const lrt_options* opt,
                                     lrt_ctx** out) {
  if (!out) return bad("out is NULL");
  *out = nullptr;
  if (!cell || !kmesh || !q || !nG || !omega || !kernel) return bad("NULL argument");
  if (cell->natoms < 1 || !cell->positions) return bad("natoms must be >= 1 with positions");
  if (!(cell->Z > 0) || !(cell->ecut > 0) || !(cell->r_c >= 0)) return bad("Z, ecut, r_c");
  if (cell->potential != LRT_POT_EMPTY_CORE && cell->potential != LRT_POT_ZERO)
    return bad("unknown potential kind");
  if (cell->basis != LRT_BASIS_SPHERE && cell->basis != LRT_BASIS_FIXED)
    return bad("unknown basis kind");
  for (int i = 0; i < 3; ++i)
    if (kmesh->n[i] < 1 || kmesh->n[i] > 256) return bad("k mesh size");
  if (kmesh->scheme != LRT_K_COMMENSURATE && kmesh->scheme != LRT_K_TR_SYMMETRIC)
    return bad("unknown k scheme");
  if (nbands < 1) return bad("nbands must be >= 1");
  if (!(T > 0) || !std::isfinite(T)) return bad("T must be > 0");
  if (!(eta > 0) || !std::isfinite(eta)) return bad("eta must be > 0");
  if (nq < 1) return bad("nq must be >= 1");
  if (nw < 2) return bad("nw must be >= 2");
  for (int j = 0; j < nw; ++j)
    if (!std::isfinite(omega[j]) || (j > 0 && !(omega[j] > omega[j - 1])))
      return bad("omega must be finite and strictly increasing");
  for (int i = 0; i < 3 * nq; ++i)
    if (!std::isfinite(q[i])) return bad("q must be finite");
  for (int i = 0; i < nq; ++i)
    if (nG[i] < 1 || nG[i] > 4096) return bad("nG out of range");
  if (kernel->kind < LRT_KERNEL_RPA || kernel->kind > LRT_KERNEL_FXC_MODEL)
    return bad("unknown kernel kind");
  lrt_options o{LRT_PREC_FP64, 0, 0};
  if (opt) o = *opt;
  if (o.precision < LRT_PREC_FP64 || o.precision > LRT_PREC_BF16X3) return bad("precision");

  lrt_ctx* c = new (std::nothrow) lrt_ctx();
  if (!c) {
    set_error("host allocation");
    return LRT_ENOMEM;
  }
  std::memcpy(c->lattice, cell->lattice, sizeof(c->lattice));
  c->natoms = cell->natoms;
  c->positions.assign(cell->positions, cell->positions + 3 * cell->natoms);
  c->Z = cell->Z;
  c->r_c = cell->r_c;
  c->ecut = cell->ecut;
  c->potential = cell->potential;
  c->basis = cell->basis;
  for (int i = 0; i < 3; ++i) c->kn[i] = kmesh->n[i];
  c->kscheme = kmesh->scheme;
  c->nk = c->kn[0] * c->kn[1] * c->kn[2];
  c->nbands = nbands;
  c->nb = nbands;
  c->T = T;
  c->eta = eta;
  c->etas.assign(1, eta);
  c->neta = 1;
  c->nq = nq;
  c->q.assign(q, q + 3 * nq);
  c->nw = nw;
  c->omega.assign(omega, omega + nw);
  c->kernel = *kernel;
  c->precision = o.precision;
  c->device = o.device;
  c->np = (int64_t)c->nk * c->nb * c->nb;
  // internal frequencies: the grid, plus w = 0 when it is not on it (S(q,0) enters Eq. 1)
  c->freqs = c->omega;
  c->hcol = -1;
  for (int j = 0; j < nw; ++j)
    if (c->omega[j] == 0.0) {
      c->hcol = j;
      break;
    }
  if (c->hcol < 0) {
    c->freqs.push_back(0.0);
    c->hcol = nw;
  }
  c->nwi = (int)c->freqs.size();

  c->host_only = (o.flags & LRT_FLAG_HOST_ONLY) != 0;
  lrt_status st = [&]() -> lrt_status {
    LRT_TRY(build_geometry(c, nG));
    if (2.0 * c->nb < c->nelec) return bad("not enough bands to hold the electrons");
    if (c->host_only) return LRT_OK;
    LRT_CUDA(cudaSetDevice(c->device));
    LRT_TRY(solve_ground_states(c, occupations));
    for (auto& Q : c->qd) {
      LRT_CUDA(cudaMalloc(&Q.Kdev, Q.nG * sizeof(double)));
      LRT_CUDA(cudaMemcpy(Q.Kdev, Q.K.data(), Q.nG * sizeof(double), cudaMemcpyHostToDevice));
    }
    LRT_CUDA(cudaMalloc(&c->dw.delta, c->np * sizeof(double)));
    LRT_CUDA(cudaMalloc(&c->dw.df, c->np * sizeof(double)));
    LRT_CUDA(cudaMalloc(&c->dw.freqs, c->nwi * sizeof(double)));
    LRT_CUDA(cudaMalloc(&c->dw.omega, c->nw * sizeof(double)));
    LRT_CUDA(cudaMalloc(&c->dw.S, (size_t)c->nq * c->nw * sizeof(double)));
    LRT_CUDA(cudaMalloc(&c->dw.chi00, (size_t)c->nq * c->nwi * sizeof(double2)));
    LRT_CUDA(cudaMalloc(&c->dw.status, sizeof(int)));
    LRT_CUDA(cudaMemset(c->dw.status, 0, sizeof(int)));
    LRT_CUDA(cudaMemcpy(c->dw.freqs, c->freqs.data(), c->nwi * sizeof(double),
                        cudaMemcpyHostToDevice));
    LRT_CUDA(cudaMemcpy(c->dw.omega, c->omega.data(), c->nw * sizeof(double),
                        cudaMemcpyHostToDevice));
    return LRT_OK;
  }();
  if (st != LRT_OK) {
    free_ctx(c);
    return st;
  }
  *out = c;
  return LRT_OK;
}

extern "C" lrt_status lrtddft_destroy(lrt_ctx* ctx) {
  free_ctx(ctx);
  return LRT_OK;
}

extern "C" lrt_status lrtddft_query(const lrt_ctx* c, int64_t out[8]) {
  if (!c || !out) return bad("NULL argument");
  out[0] = c->nq;
  out[1] = c->nw;
  out[2] = c->nk;
  out[3] = c->nb;
  out[4] = c->nGmax;
  out[5] = c->npw;
  out[6] = c->nwi;
  out[7] = c->precision;
  return LRT_OK;
}

static lrt_status need_device(const lrt_ctx* c) {
  if (c->host_only) {
    set_error("host-only context");
    return LRT_ESTATE;
  }
  LRT_CUDA(cudaSetDevice(c->device));
  return LRT_OK;
}

extern "C" lrt_status lrtddft_chi0_assemble(lrt_ctx* c, int q_begin, int q_end, void* stream) {
  if (!c) return bad("NULL context");
  LRT_TRY(need_device(c));
  if (q_begin < 0 || q_end > c->nq || q_begin >= q_end) return bad("q range");
  cudaStream_t s = (cudaStream_t)stream;
  LRT_CUDA(cudaSetDevice(c->device));
  for (int iq = q_begin; iq < q_end; ++iq) {
    QData& Q = c->qd[iq];
    LRT_TRY(adopt_orbitals(c, iq, s));
    if (!Q.chi0) LRT_CUDA(cudaMalloc(&Q.chi0, (size_t)ncol(c) * Q.nG * Q.nG * sizeof(double2)));
  }
  LRT_TRY(ensure_zf(c));
  if (c->spectral_order) {
    // spectral engine, q by q on the shared pair-density buffer; S(q,0) from the same
    // pair densities while they are resident
    LRT_TRY(ensure_rho(c));
    const bool fp64 = c->precision == LRT_PREC_FP64;
    for (int iq = q_begin; iq < q_end; ++iq) {
      QData& Q = c->qd[iq];
      float sB = 1.0f;
      if (fp64)
        LRT_TRY(launch_pair_weights(c, Q, s));
      else
        LRT_TRY(split_pair_weights(c, Q, &sB, s));
      LRT_TRY(launch_pair_density(c, Q, c->dw.rho, !fp64, s));
      LRT_TRY(launch_chi0_spectral(c, Q, c->dw.rho, s));
      LRT_TRY(launch_s0(c, Q, iq, c->dw.rho, fp64 ? nullptr : Q.sp.pw, sB, s));
    }
  } else if (c->precision == LRT_PREC_FP64) {
    LRT_TRY(ensure_rho(c));
    for (int iq = q_begin; iq < q_end; ++iq) {
      QData& Q = c->qd[iq];
      LRT_TRY(launch_pair_weights(c, Q, s));
      LRT_TRY(launch_pair_density(c, Q, c->dw.rho, false, s));
      LRT_TRY(launch_chi0_fp64(c, Q, s));
      // S(q,0) needs this q's pair densities: before the next q overwrites them
      LRT_TRY(launch_s0(c, Q, iq, c->dw.rho, nullptr, 1.0f, s));
    }
  } else {
    LRT_TRY(launch_chi0_split_range(c, q_begin, q_end, s));
  }
  for (int iq = q_begin; iq < q_end; ++iq) {
    QData& Q = c->qd[iq];
    Q.have_chi0 = true;
    Q.have_chi = false;
    Q.have_dchi = false;
  }
  c->have_S = false;
  return LRT_OK;
}

extern "C" lrt_status lrtddft_dyson_solve(lrt_ctx* c, int q_begin, int q_end, void* stream) {
  if (!c) return bad("NULL context");
  LRT_TRY(need_device(c));
  if (q_begin < 0 || q_end > c->nq || q_begin >= q_end) return bad("q range");
  cudaStream_t s = (cudaStream_t)stream;
  LRT_CUDA(cudaSetDevice(c->device));
  for (int iq = q_begin; iq < q_end; ++iq) {
    QData& Q = c->qd[iq];
    if (!Q.have_chi0) {
      set_error("dyson_solve before chi0_assemble");
      return LRT_ESTATE;
    }
    if (!Q.chi) LRT_CUDA(cudaMalloc(&Q.chi, (size_t)ncol(c) * Q.nG * sizeof(double2)));
    LRT_TRY(launch_dyson(c, Q, iq, s));
    Q.have_chi = true;
    Q.have_dchi = false;
  }
  c->have_S = false;
  return LRT_OK;
}

static lrt_status apply_eta_list(lrt_ctx* c, int n, const double* etas);
static lrt_status check_tau(const lrt_ctx* c, int ntau, const double* tau);

static lrt_status need_all_chi(lrt_ctx* c) {
  LRT_TRY(need_device(c));
  for (auto& Q : c->qd)
    if (!Q.have_chi) {
      set_error("spectra requested before dyson_solve on every q");
      return LRT_ESTATE;
    }
  return LRT_OK;
}

extern "C" lrt_status lrtddft_dsf_device(lrt_ctx* c, double* S_dev, void* stream) {
  if (!c || !S_dev) return bad("NULL argument");
  LRT_TRY(need_all_chi(c));
  LRT_TRY(launch_dsf(c, S_dev, (cudaStream_t)stream));
  return LRT_OK;
}

extern "C" lrt_status lrtddft_dsf(lrt_ctx* c, double* S) {
  if (!c || !S) return bad("NULL argument");
  LRT_TRY(need_all_chi(c));
  // host-buffer calls run on the legacy stream after all earlier work on any stream
  LRT_CUDA(cudaDeviceSynchronize());
  LRT_TRY(launch_dsf(c, c->dw.S, 0));
  LRT_CUDA(cudaMemcpy(S, c->dw.S, (size_t)nrow(c) * c->nw * sizeof(double), cudaMemcpyDeviceToHost));
  LRT_TRY(check_status_word(c));
  c->have_S = true;
  return LRT_OK;
}

extern "C" lrt_status lrtddft_itcf_laplace_device(lrt_ctx* c, int ntau, const double* tau_dev,
                                                  int mode, double* F_dev, double* metrics_dev,
                                                  void* stream) {
  if (!c || !tau_dev || !F_dev) return bad("NULL argument");
  if (ntau < 1) return bad("ntau must be >= 1");
  if (mode != LRT_ITCF_FOLD && mode != LRT_ITCF_DIRECT) return bad("unknown ITCF mode");
  LRT_TRY(need_all_chi(c));
  cudaStream_t s = (cudaStream_t)stream;
  LRT_TRY(launch_dsf(c, c->dw.S, s));
  LRT_TRY(launch_itcf(c, c->dw.S, ntau, tau_dev, mode, F_dev, metrics_dev, s));
  return LRT_OK;
}

extern "C" lrt_status lrtddft_itcf_laplace(lrt_ctx* c, int ntau, const double* tau, int mode,
                                           double* F, double* metrics) {
  if (!c || !tau || !F) return bad("NULL argument");
  if (ntau < 1) return bad("ntau must be >= 1");
  for (int i = 0; i < ntau; ++i)
    if (!(tau[i] >= 0.0) || tau[i] > 1.0 / c->T * (1.0 + 1e-12)) return bad("tau outside [0, beta]");
  LRT_TRY(need_device(c));
  double *dtau = nullptr, *dF = nullptr, *dm = nullptr;
  auto done = [&](lrt_status st) {
    cudaFree(dtau);
    cudaFree(dF);
    cudaFree(dm);
    return st;
  };
  if (cudaMalloc(&dtau, ntau * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dF, (size_t)nrow(c) * ntau * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dm, (size_t)nrow(c) * 5 * sizeof(double)) != cudaSuccess) {
    set_error("device allocation");
    return done(LRT_ENOMEM);
  }
  if (cudaMemcpy(dtau, tau, ntau * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess)
    return done(LRT_ECUDA);
  lrt_status st = lrtddft_itcf_laplace_device(c, ntau, dtau, mode, dF, dm, 0);
  if (st != LRT_OK) return done(st);
  if (cudaMemcpy(F, dF, (size_t)nrow(c) * ntau * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return done(LRT_ECUDA);
  if (metrics &&
      cudaMemcpy(metrics, dm, (size_t)nrow(c) * 5 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return done(LRT_ECUDA);
  return done(check_status_word(c));
}

extern "C" lrt_status lrtddft_attenuate(lrt_ctx* c, const lrt_atten_params* p, double* Sp,
                                        lrt_atten_report* rep) {
  if (!c || !Sp) return bad("NULL argument");
  LRT_TRY(need_all_chi(c));
  LRT_CUDA(cudaDeviceSynchronize());
  LRT_TRY(launch_dsf(c, c->dw.S, 0));
  LRT_TRY(run_attenuation(c, p, c->dw.S, Sp, rep, 0));
  return check_status_word(c);
}

extern "C" lrt_status lrtddft_set_orbitals(lrt_ctx* c, int iq, const double* eps,
                                           const double* coeff, const double* occ) {
  if (!c || !eps || !coeff) return bad("NULL argument");
  if (iq < 0 || iq >= c->nq) return bad("q index");
  LRT_TRY(need_device(c));
  LRT_CUDA(cudaSetDevice(c->device));
  QData& Q = c->qd[iq];
  if (Q.up.pending) {
    // the later call wins: an asynchronous upload still waiting for adoption is dropped
    LRT_CUDA(cudaEventSynchronize(Q.up.ready));
    Q.up.pending = false;
  }
  size_t ne = (size_t)2 * c->nk * c->nb;
  LRT_CUDA(cudaMemcpy(Q.eps, eps, ne * sizeof(double), cudaMemcpyHostToDevice));
  LRT_CUDA(cudaMemcpy(Q.coeff, coeff, ne * c->npw * sizeof(double2), cudaMemcpyHostToDevice));
  LRT_TRY(reset_band_weights(c, iq, eps));
  if (occ) {
    Q.mu = NAN;
    LRT_CUDA(cudaMemcpy(Q.occ, occ, ne * sizeof(double), cudaMemcpyHostToDevice));
  } else {
    LRT_TRY(set_occupations_fd(c, iq, eps));
  }
  Q.have_chi0 = Q.have_chi = Q.have_dchi = false;
  c->have_S = false;
  c->graph_valid = false;
  return LRT_OK;
}

// Swap in the orbitals of a completed or in-flight lrtddft_set_orbitals_async upload of q: the
// stream s waits for the copies, the two buffer sets trade places, and the set just retired is
// marked free once the work already on s (which may still read it) is done.
namespace lrt {
lrt_status adopt_orbitals(lrt_ctx* c, int iq, cudaStream_t s) {
  QData& Q = c->qd[iq];
  if (!Q.up.pending) return LRT_OK;
  LRT_CUDA(cudaStreamWaitEvent(s, Q.up.ready, 0));
  std::swap(Q.coeff, Q.up.coeff);
  std::swap(Q.eps, Q.up.eps);
  std::swap(Q.occ, Q.up.occ);
  std::swap(Q.wgt, Q.up.wgt);
  std::swap(Q.wgt_h, Q.up.wgt_h);
  std::swap(Q.mu, Q.up.mu);
  LRT_CUDA(cudaEventRecord(Q.up.free, s));
  Q.up.pending = false;
  Q.have_chi0 = Q.have_chi = Q.have_dchi = false;
  c->have_S = false;
  c->graph_valid = false;
  return LRT_OK;
}
}  // namespace lrt

extern "C" lrt_status lrtddft_set_orbitals_async(lrt_ctx* c, int iq, const double* eps,
                                                 const double* coeff, const double* occ) {
  if (!c || !eps || !coeff) return bad("NULL argument");
  if (iq < 0 || iq >= c->nq) return bad("q index");
  LRT_TRY(need_device(c));
  LRT_CUDA(cudaSetDevice(c->device));
  QData& Q = c->qd[iq];
  auto& U = Q.up;
  const size_t ne = (size_t)2 * c->nk * c->nb;
  const size_t nc = ne * c->npw;
  if (!c->upload) LRT_CUDA(cudaStreamCreateWithFlags(&c->upload, cudaStreamNonBlocking));
  if (!U.coeff) {
    LRT_CUDA(cudaMalloc(&U.coeff, nc * sizeof(double2)));
    LRT_CUDA(cudaMalloc(&U.eps, ne * sizeof(double)));
    LRT_CUDA(cudaMalloc(&U.occ, ne * sizeof(double)));
    LRT_CUDA(cudaMalloc(&U.wgt, ne * sizeof(double)));
    LRT_CUDA(cudaMallocHost(&U.stage, 3 * ne * sizeof(double)));
    LRT_CUDA(cudaEventCreateWithFlags(&U.ready, cudaEventDisableTiming));
    LRT_CUDA(cudaEventCreateWithFlags(&U.free, cudaEventDisableTiming));
    U.wgt_h.assign(ne, 0.0);
  }
  // an earlier upload into these buffers may still be reading the staging area
  LRT_CUDA(cudaEventSynchronize(U.ready));
  double* st_eps = U.stage;
  double* st_occ = U.stage + ne;
  double* st_wgt = U.stage + 2 * ne;
  std::copy(eps, eps + ne, st_eps);
  LRT_TRY(band_weights_all(c, eps, U.wgt_h.data()));
  std::copy(U.wgt_h.begin(), U.wgt_h.end(), st_wgt);
  if (occ) {
    U.mu = NAN;
    std::copy(occ, occ + ne, st_occ);
  } else {
    LRT_TRY(fermi_occupations(c, eps, U.wgt_h.data(), st_occ, &U.mu));
  }
  // the buffers about to be written were read by work enqueued before the last swap
  LRT_CUDA(cudaStreamWaitEvent(c->upload, U.free, 0));
  LRT_CUDA(cudaMemcpyAsync(U.coeff, coeff, nc * sizeof(double2), cudaMemcpyHostToDevice, c->upload));
  LRT_CUDA(cudaMemcpyAsync(U.eps, st_eps, ne * sizeof(double), cudaMemcpyHostToDevice, c->upload));
  LRT_CUDA(cudaMemcpyAsync(U.occ, st_occ, ne * sizeof(double), cudaMemcpyHostToDevice, c->upload));
  LRT_CUDA(cudaMemcpyAsync(U.wgt, st_wgt, ne * sizeof(double), cudaMemcpyHostToDevice, c->upload));
  LRT_CUDA(cudaEventRecord(U.ready, c->upload));
  U.pending = true;
  return LRT_OK;
}

extern "C" lrt_status lrtddft_get_basis(const lrt_ctx* c, int iq, int32_t* miller, int32_t* npw_k) {
  if (!c || !miller || !npw_k) return bad("NULL argument");
  if (iq < 0 || iq >= c->nq) return bad("q index");
  const QData& Q = c->qd[iq];
  std::copy(Q.miller.begin(), Q.miller.end(), miller);
  std::copy(Q.npw_k.begin(), Q.npw_k.end(), npw_k);
  return LRT_OK;
}

extern "C" lrt_status lrtddft_get_ground_state(const lrt_ctx* c, int iq, double* eps, double* occ,
                                               double* weights, double* mu) {
  if (!c) return bad("NULL context");
  if (iq < 0 || iq >= c->nq) return bad("q index");
  LRT_TRY(need_device(c));
  LRT_TRY(adopt_orbitals(const_cast<lrt_ctx*>(c), iq, 0));
  const QData& Q = c->qd[iq];
  size_t ne = (size_t)2 * c->nk * c->nb;
  if (eps) LRT_CUDA(cudaMemcpy(eps, Q.eps, ne * sizeof(double), cudaMemcpyDeviceToHost));
  if (occ) LRT_CUDA(cudaMemcpy(occ, Q.occ, ne * sizeof(double), cudaMemcpyDeviceToHost));
  if (weights) std::copy(Q.wgt_h.begin(), Q.wgt_h.end(), weights);
  if (mu) *mu = Q.mu;
  return LRT_OK;
}

extern "C" lrt_status lrtddft_get_gset(const lrt_ctx* c, int iq, int32_t* miller, double* K) {
  if (!c) return bad("NULL context");
  if (iq < 0 || iq >= c->nq) return bad("q index");
  const QData& Q = c->qd[iq];
  if (miller) std::copy(Q.gset.begin(), Q.gset.end(), miller);
  if (K) std::copy(Q.K.begin(), Q.K.end(), K);
  return LRT_OK;
}

extern "C" lrt_status lrtddft_get_chi0(const lrt_ctx* c, int iq, double* chi0) {
  if (!c || !chi0) return bad("NULL argument");
  if (iq < 0 || iq >= c->nq) return bad("q index");
  const QData& Q = c->qd[iq];
  if (!Q.have_chi0) {
    set_error("get_chi0 before chi0_assemble");
    return LRT_ESTATE;
  }
  LRT_CUDA(cudaMemcpy(chi0, Q.chi0, (size_t)ncol(c) * Q.nG * Q.nG * sizeof(double2),
                      cudaMemcpyDeviceToHost));
  return LRT_OK;
}

extern "C" lrt_status lrtddft_get_chi_col0(const lrt_ctx* c, int iq, double* chi) {
  if (!c || !chi) return bad("NULL argument");
  if (iq < 0 || iq >= c->nq) return bad("q index");
  const QData& Q = c->qd[iq];
  if (!Q.have_chi) {
    set_error("get_chi_col0 before dyson_solve");
    return LRT_ESTATE;
  }
  LRT_CUDA(cudaMemcpy(chi, Q.chi, (size_t)ncol(c) * Q.nG * sizeof(double2), cudaMemcpyDeviceToHost));
  return LRT_OK;
}

extern "C" lrt_status lrtddft_get_frequencies(const lrt_ctx* c, double* freqs, int* hcol) {
  if (!c) return bad("NULL context");
  if (freqs) std::copy(c->freqs.begin(), c->freqs.end(), freqs);
  if (hcol) *hcol = c->hcol;
  return LRT_OK;
}

static void drop_events(const lrt_ctx* c) {
  for (auto& e : c->ev_chi0) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto& e : c->ev_rho) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  c->ev_chi0.clear();
  c->ev_rho.clear();
}

extern "C" lrt_status lrtddft_profile(lrt_ctx* c, int enable) {
  if (!c) return bad("NULL context");
  LRT_TRY(need_device(c));
  LRT_CUDA(cudaDeviceSynchronize());
  drop_events(c);
  c->launches = 0;
  c->timed_cmac = 0.0;
  c->profiling = enable != 0;
  return LRT_OK;
}

extern "C" lrt_status lrtddft_profile_read(lrt_ctx* c, double out[8]) {
  if (!c || !out) return bad("NULL argument");
  LRT_TRY(need_device(c));
  LRT_CUDA(cudaDeviceSynchronize());
  double t_chi0 = 0.0, t_rho = 0.0;
  for (auto& e : c->ev_chi0) {
    float ms = 0.f;
    LRT_CUDA(cudaEventElapsedTime(&ms, e.first, e.second));
    t_chi0 += ms;
  }
  for (auto& e : c->ev_rho) {
    float ms = 0.f;
    LRT_CUDA(cudaEventElapsedTime(&ms, e.first, e.second));
    t_rho += ms;
  }
  out[0] = (double)c->launches;
  out[1] = (double)c->ev_chi0.size();
  out[2] = t_chi0;
  out[3] = (double)c->ev_rho.size();
  out[4] = t_rho;
  out[5] = c->timed_cmac;
  out[6] = out[7] = 0.0;
  return LRT_OK;
}

extern "C" lrt_status lrtddft_get_orbitals(const lrt_ctx* c, int iq, double* coeff) {
  if (!c || !coeff) return bad("NULL argument");
  if (iq < 0 || iq >= c->nq) return bad("q index");
  LRT_TRY(need_device(c));
  LRT_TRY(adopt_orbitals(const_cast<lrt_ctx*>(c), iq, 0));
  const QData& Q = c->qd[iq];
  LRT_CUDA(cudaMemcpy(coeff, Q.coeff, (size_t)2 * c->nk * c->nb * c->npw * sizeof(double2),
                      cudaMemcpyDeviceToHost));
  return LRT_OK;
}

// ------------------------------------------------------------------ parameters and adjoint

extern "C" lrt_status lrtddft_set_params(lrt_ctx* c, double T, double eta, const lrt_kernel* kernel) {
  if (!c || !kernel) return bad("NULL argument");
  if (!(T > 0) || !std::isfinite(T)) return bad("T must be > 0");
  if (!(eta > 0) || !std::isfinite(eta)) return bad("eta must be > 0");
  if (kernel->kind < LRT_KERNEL_RPA || kernel->kind > LRT_KERNEL_FXC_MODEL)
    return bad("unknown kernel kind");
  if (!std::isfinite(kernel->A) || !std::isfinite(kernel->B) || !std::isfinite(kernel->C))
    return bad("kernel parameters must be finite");
  LRT_TRY(need_device(c));
  LRT_CUDA(cudaSetDevice(c->device));
  LRT_CUDA(cudaDeviceSynchronize());
  LRT_TRY(apply_eta_list(c, 1, &eta));
  c->T = T;
  c->kernel = *kernel;
  c->graph_valid = false;
  const size_t ne = (size_t)2 * c->nk * c->nb;
  std::vector<double> eps(ne);
  for (int iq = 0; iq < c->nq; ++iq) {
    QData& Q = c->qd[iq];
    LRT_TRY(adopt_orbitals(c, iq, 0));
    kernel_diag(c, Q);
    LRT_CUDA(cudaMemcpy(Q.Kdev, Q.K.data(), Q.nG * sizeof(double), cudaMemcpyHostToDevice));
    if (!std::isnan(Q.mu)) {   // Fermi-Dirac occupations (not supplied by the caller)
      LRT_CUDA(cudaMemcpy(eps.data(), Q.eps, ne * sizeof(double), cudaMemcpyDeviceToHost));
      LRT_TRY(set_occupations_fd(c, iq, eps.data()));
    }
    Q.have_chi0 = Q.have_chi = Q.have_dchi = false;
  }
  c->have_S = false;
  return LRT_OK;
}

// Install an eta list (ascending, validated by the caller): everything sized by the number of
// chi0 columns or spectrum rows is released or reallocated, and chi0, chi and the plans of
// the tensor path are dropped (they are rebuilt by the next assemble).
static lrt_status apply_eta_list(lrt_ctx* c, int n, const double* etas) {
  const bool same_size = n == c->neta;
  c->etas.assign(etas, etas + n);
  c->neta = n;
  c->eta = etas[0];
  c->graph_valid = false;
  c->have_S = false;
  for (auto& Q : c->qd) {
    Q.have_chi0 = Q.have_chi = Q.have_dchi = false;
    if (!same_size) {
      cudaFree(Q.chi0);
      cudaFree(Q.chi);
      Q.chi0 = Q.chi = nullptr;
    }
    free_split_plan(Q.sp);   // the column tables carry the etas
  }
  if (same_size) return LRT_OK;
  cudaFree(c->dw.S);
  cudaFree(c->dw.chi00);
  cudaFree(c->dw.s0);
  cudaFree(c->dw.eta_ref);
  c->dw.S = nullptr;
  c->dw.s0 = nullptr;
  c->dw.chi00 = nullptr;
  c->dw.eta_ref = nullptr;
  LRT_CUDA(cudaMalloc(&c->dw.S, (size_t)nrow(c) * c->nw * sizeof(double)));
  LRT_CUDA(cudaMalloc(&c->dw.chi00, (size_t)c->nq * ncol(c) * sizeof(double2)));
  LRT_CUDA(cudaMalloc(&c->dw.s0, (size_t)nrow(c) * sizeof(double2)));
  LRT_CUDA(cudaMemset(c->dw.s0, 0, (size_t)nrow(c) * sizeof(double2)));
  return LRT_OK;
}

extern "C" lrt_status lrtddft_set_eta_list(lrt_ctx* c, int n_eta, const double* eta) {
  if (!c || !eta) return bad("NULL argument");
  if (n_eta < 1 || n_eta > 64) return bad("n_eta must be in 1..64");
  for (int j = 0; j < n_eta; ++j)
    if (!(eta[j] > 0) || !std::isfinite(eta[j]) || (j > 0 && !(eta[j] > eta[j - 1])))
      return bad("etas must be positive, finite and strictly increasing");
  LRT_TRY(need_device(c));
  LRT_CUDA(cudaDeviceSynchronize());
  return apply_eta_list(c, n_eta, eta);
}

extern "C" lrt_status lrtddft_get_eta_list(const lrt_ctx* c, int* n_eta, double* eta) {
  if (!c || !n_eta) return bad("NULL argument");
  *n_eta = c->neta;
  if (eta) std::copy(c->etas.begin(), c->etas.end(), eta);
  return LRT_OK;
}

extern "C" lrt_status lrtddft_eta_scan(lrt_ctx* c, int ntau, const double* tau, double tol, double* F,
                                       double* metrics, int* eta_ref) {
  if (!c || !tau || !eta_ref) return bad("NULL argument");
  if (!(tol >= 0) || !std::isfinite(tol)) return bad("tol must be finite and >= 0");
  LRT_TRY(check_tau(c, ntau, tau));
  LRT_TRY(need_all_chi(c));
  LRT_CUDA(cudaDeviceSynchronize());
  if (!c->dw.eta_ref) LRT_CUDA(cudaMalloc(&c->dw.eta_ref, (size_t)c->nq * sizeof(int)));
  double *dtau = nullptr, *dF = nullptr, *dm = nullptr;
  auto done = [&](lrt_status st) {
    cudaFree(dtau);
    cudaFree(dF);
    cudaFree(dm);
    return st;
  };
  if (cudaMalloc(&dtau, ntau * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dF, (size_t)nrow(c) * ntau * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dm, (size_t)nrow(c) * 5 * sizeof(double)) != cudaSuccess) {
    set_error("device allocation");
    return done(LRT_ENOMEM);
  }
  if (cudaMemcpy(dtau, tau, ntau * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return done(LRT_ECUDA);
  lrt_status st = launch_dsf(c, c->dw.S, 0);
  if (st == LRT_OK) st = launch_itcf(c, c->dw.S, ntau, dtau, LRT_ITCF_FOLD, dF, dm, 0);
  if (st == LRT_OK) st = launch_eta_pick(c, dm, c->nq, c->neta, tol, c->dw.eta_ref, 0);
  if (st != LRT_OK) return done(st);
  if ((F && cudaMemcpy(F, dF, (size_t)nrow(c) * ntau * sizeof(double), cudaMemcpyDeviceToHost) !=
                cudaSuccess) ||
      (metrics && cudaMemcpy(metrics, dm, (size_t)nrow(c) * 5 * sizeof(double),
                             cudaMemcpyDeviceToHost) != cudaSuccess) ||
      cudaMemcpy(eta_ref, c->dw.eta_ref, (size_t)c->nq * sizeof(int), cudaMemcpyDeviceToHost) !=
          cudaSuccess)
    return done(LRT_ECUDA);
  return done(check_status_word(c));
}

// d chi_00/d theta of every q (cached until chi0, chi or the parameters change)
static lrt_status ensure_dchi(lrt_ctx* c) {
  if (c->neta > 1) {
    set_error("the adjoint takes a single eta (set_params or an eta list of one)");
    return LRT_EUNSUPPORTED;
  }
  if (c->spectral_order) {
    set_error("the adjoint differentiates the direct pair sum; use the direct chi0 engine");
    return LRT_EUNSUPPORTED;
  }
  LRT_TRY(need_all_chi(c));
  LRT_CUDA(cudaSetDevice(c->device));
  LRT_CUDA(cudaDeviceSynchronize());
  bool any = false;
  for (auto& Q : c->qd) any = any || !Q.have_dchi;
  if (!any) return LRT_OK;
  LRT_TRY(ensure_rho(c));
  for (int iq = 0; iq < c->nq; ++iq) {
    QData& Q = c->qd[iq];
    if (Q.have_dchi) continue;
    LRT_TRY(launch_pair_density(c, Q, c->dw.rho, c->precision != LRT_PREC_FP64, 0));
    LRT_TRY(launch_adjoint_q(c, Q, iq, Q.dchi, 0));
    LRT_TRY(check_status_word(c));
    Q.have_dchi = true;
  }
  return LRT_OK;
}

// S of q iq on the caller's grid and dS/dtheta [nw][5] (Eq. 8 and its w -> 0 form)
static lrt_status s_and_jacobian(lrt_ctx* c, int iq, std::vector<double>& S, std::vector<double>& dS,
                                 double& S0, double dS0[5]) {
  const QData& Q = c->qd[iq];
  std::vector<double2> chi00(c->nwi);
  LRT_CUDA(cudaMemcpy2D(chi00.data(), sizeof(double2), Q.chi, (size_t)Q.nG * sizeof(double2),
                        sizeof(double2), c->nwi, cudaMemcpyDeviceToHost));
  const double beta = 1.0 / c->T, pin = M_PI * c->density;
  auto dim = [&](int w, int j) { return Q.dchi[(size_t)w * 10 + 2 * j + 1]; };
  S.assign(c->nw, 0.0);
  dS.assign((size_t)c->nw * 5, 0.0);
  // w -> 0: S(0) = (T/(pi n)) Re s, s = d chi_00/d eta (the eta tangent at w = 0), and its
  // tangents from the second-order pieces d s/d theta
  const double s_re = Q.dchi[(size_t)c->hcol * 10 + 2];
  S0 = c->T * s_re / pin;
  for (int j = 0; j < 5; ++j) dS0[j] = c->T * Q.ds0[2 * j] / pin;
  dS0[0] += s_re / pin;
  for (int w = 0; w < c->nw; ++w) {
    const double om = c->omega[w];
    if (om == 0.0) {
      S[w] = S0;
      for (int j = 0; j < 5; ++j) dS[(size_t)w * 5 + j] = dS0[j];
      continue;
    }
    const double g = 1.0 / (-std::expm1(-beta * om));
    S[w] = -chi00[w].y * g / pin;
    for (int j = 0; j < 5; ++j) dS[(size_t)w * 5 + j] = -dim(w, j) * g / pin;
    // d/dT of 1/(1 - e^{-w/T})
    const double dg = std::exp(-beta * om) * om / (c->T * c->T) * g * g;
    dS[(size_t)w * 5] += -chi00[w].y * dg / pin;
  }
  return LRT_OK;
}

static lrt_status check_tau(const lrt_ctx* c, int ntau, const double* tau) {
  if (ntau < 1) return bad("ntau must be >= 1");
  for (int i = 0; i < ntau; ++i)
    if (!(tau[i] >= 0.0) || tau[i] > 1.0 / c->T * (1.0 + 1e-12)) return bad("tau outside [0, beta]");
  return LRT_OK;
}

// dF/dtheta [ntau][5] of q iq (FOLD form of Eq. 1 at fixed absolute tau)
static void f_jacobian(const lrt_ctx* c, const std::vector<double>& S, const std::vector<double>& dS,
                       double S0, const double dS0[5], int ntau, const double* tau, double* dF) {
  // positive branch: w >= 0 in grid order, with w = 0 prepended (value S0) when absent
  std::vector<double> wp, sp, dsp;
  for (int w = 0; w < c->nw; ++w)
    if (c->omega[w] >= 0.0) {
      if (wp.empty() && c->omega[w] != 0.0) {
        wp.push_back(0.0);
        sp.push_back(S0);
        for (int j = 0; j < 5; ++j) dsp.push_back(dS0[j]);
      }
      wp.push_back(c->omega[w]);
      sp.push_back(S[w]);
      for (int j = 0; j < 5; ++j) dsp.push_back(dS[(size_t)w * 5 + j]);
    }
  if (wp.empty()) {
    wp.push_back(0.0);
    sp.push_back(S0);
    for (int j = 0; j < 5; ++j) dsp.push_back(dS0[j]);
  }
  const size_t m = wp.size();
  std::vector<double> wt(m, 0.0);
  for (size_t i = 0; i + 1 < m; ++i) {
    const double dx = wp[i + 1] - wp[i];
    wt[i] += 0.5 * dx;
    wt[i + 1] += 0.5 * dx;
  }
  const double beta = 1.0 / c->T;
  for (int t = 0; t < ntau; ++t) {
    double acc[5] = {0, 0, 0, 0, 0};
    for (size_t i = 0; i < m; ++i) {
      const double e1 = std::exp(-tau[t] * wp[i]), e2 = std::exp(-(beta - tau[t]) * wp[i]);
      for (int j = 0; j < 5; ++j) acc[j] += wt[i] * (e1 + e2) * dsp[i * 5 + j];
      acc[0] += wt[i] * sp[i] * wp[i] * e2 / (c->T * c->T);
    }
    for (int j = 0; j < 5; ++j) dF[(size_t)t * 5 + j] = acc[j];
  }
}

extern "C" lrt_status lrtddft_jacobian(lrt_ctx* c, int ntau, const double* tau, double* dS,
                                       double* dF) {
  if (!c || (!dS && !dF)) return bad("NULL argument");
  if (dF) {
    if (!tau) return bad("NULL argument");
    LRT_TRY(check_tau(c, ntau, tau));
  }
  LRT_TRY(ensure_dchi(c));
  std::vector<double> S, J;
  double S0, dS0[5];
  for (int iq = 0; iq < c->nq; ++iq) {
    LRT_TRY(s_and_jacobian(c, iq, S, J, S0, dS0));
    if (dS) std::copy(J.begin(), J.end(), dS + (size_t)iq * c->nw * 5);
    if (dF) f_jacobian(c, S, J, S0, dS0, ntau, tau, dF + (size_t)iq * ntau * 5);
  }
  return LRT_OK;
}

extern "C" lrt_status lrtddft_itcf_vjp(lrt_ctx* c, int ntau, const double* tau, const double* dL_dF,
                                       double grad[5]) {
  if (!c || !tau || !dL_dF || !grad) return bad("NULL argument");
  LRT_TRY(check_tau(c, ntau, tau));
  LRT_TRY(ensure_dchi(c));
  std::vector<double> S, J, jf((size_t)ntau * 5);
  double S0, dS0[5];
  for (int j = 0; j < 5; ++j) grad[j] = 0.0;
  for (int iq = 0; iq < c->nq; ++iq) {
    LRT_TRY(s_and_jacobian(c, iq, S, J, S0, dS0));
    f_jacobian(c, S, J, S0, dS0, ntau, tau, jf.data());
    for (int t = 0; t < ntau; ++t)
      for (int j = 0; j < 5; ++j) grad[j] += dL_dF[(size_t)iq * ntau + t] * jf[(size_t)t * 5 + j];
  }
  return LRT_OK;
}

extern "C" lrt_status lrtddft_dsf_vjp(lrt_ctx* c, const double* dL_dS, double grad[5]) {
  if (!c || !dL_dS || !grad) return bad("NULL argument");
  LRT_TRY(ensure_dchi(c));
  std::vector<double> S, J;
  double S0, dS0[5];
  for (int j = 0; j < 5; ++j) grad[j] = 0.0;
  for (int iq = 0; iq < c->nq; ++iq) {
    LRT_TRY(s_and_jacobian(c, iq, S, J, S0, dS0));
    for (int w = 0; w < c->nw; ++w)
      for (int j = 0; j < 5; ++j) grad[j] += dL_dS[(size_t)iq * c->nw + w] * J[(size_t)w * 5 + j];
  }
  return LRT_OK;
}

// ------------------------------------------------------------------ tuning and graphs

extern "C" lrt_status lrtddft_set_tuning(lrt_ctx* c, int flags, int variant, int unit_stages) {
  if (!c) return bad("NULL context");
  if (flags & ~(LRT_TUNE_AUTO | LRT_TUNE_SINGLE_Q | LRT_TUNE_PAIR_SIMT | LRT_TUNE_FINE_ACCUM |
                LRT_TUNE_HALF_TILES | LRT_TUNE_ZERO_SIMT))
    return bad("unknown tuning flags");
  if (variant < -1 || variant > 1) return bad("variant must be -1, 0 or 1");
  if (unit_stages != 0 && (unit_stages < 64 || unit_stages % 64 != 0))
    return bad("unit_stages must be 0 or a positive multiple of 64");
  c->autotune = (flags & LRT_TUNE_AUTO) != 0;
  c->multi_q = (flags & LRT_TUNE_SINGLE_Q) == 0;
  c->pair_simt = (flags & LRT_TUNE_PAIR_SIMT) != 0;
  c->fine_accum = (flags & LRT_TUNE_FINE_ACCUM) != 0;
  c->half_tiles = (flags & LRT_TUNE_HALF_TILES) != 0;
  c->zero_simt = (flags & LRT_TUNE_ZERO_SIMT) != 0;
  c->tune_variant = variant;
  c->tune_unit_stages = unit_stages;
  c->graph_valid = false;
  return LRT_OK;
}

extern "C" lrt_status lrtddft_get_tuning(lrt_ctx* c, int* variant, int* unit_stages) {
  if (!c || !variant || !unit_stages) return bad("NULL argument");
  *variant = c->last_tc_variant;
  *unit_stages = c->last_tc_unit_stages;
  return LRT_OK;
}

extern "C" lrt_status lrtddft_set_spectral(lrt_ctx* c, double h, int order) {
  if (!c) return bad("NULL context");
  if (h == 0.0) {
    c->spectral_order = 0;
    c->spectral_h = 0.0;
  } else {
    if (!(h > 0.0) || !std::isfinite(h)) return bad("h must be 0 or a positive bin width");
    if (order != 1 && order != 3) return bad("order must be 1 or 3");
    c->spectral_order = order;
    c->spectral_h = h;
  }
  c->graph_valid = false;
  for (auto& Q : c->qd) Q.have_chi0 = Q.have_chi = Q.have_dchi = false;
  c->have_S = false;
  return LRT_OK;
}

extern "C" lrt_status lrtddft_get_spectral_grid(const lrt_ctx* c, int iq, double* x0, long long* nbins) {
  if (!c || !x0 || !nbins) return bad("NULL argument");
  if (iq < 0 || iq >= c->nq) return bad("q index");
  *x0 = c->qd[iq].sp_x0;
  *nbins = c->qd[iq].sp_nbins;
  return LRT_OK;
}

extern "C" lrt_status lrtddft_get_tile_rows(lrt_ctx* c, int* rows) {
  if (!c || !rows) return bad("NULL argument");
  *rows = c->last_tc_rows;
  return LRT_OK;
}

static lrt_status forward_all(lrt_ctx* c, int ntau, const double* tau_dev, int mode, double* S_dev,
                              double* F_dev, double* metrics_dev, cudaStream_t s) {
  LRT_TRY(lrtddft_chi0_assemble(c, 0, c->nq, s));
  LRT_TRY(lrtddft_dyson_solve(c, 0, c->nq, s));
  LRT_TRY(lrtddft_dsf_device(c, S_dev, s));
  LRT_TRY(lrtddft_itcf_laplace_device(c, ntau, tau_dev, mode, F_dev, metrics_dev, s));
  return LRT_OK;
}

extern "C" lrt_status lrtddft_graph_capture(lrt_ctx* c, int ntau, const double* tau_dev, int mode,
                                            double* S_dev, double* F_dev, double* metrics_dev) {
  if (!c || !tau_dev || !S_dev || !F_dev || !metrics_dev) return bad("NULL argument");
  if (ntau < 1) return bad("ntau must be >= 1");
  if (mode != LRT_ITCF_FOLD && mode != LRT_ITCF_DIRECT) return bad("unknown ITCF mode");
  LRT_TRY(need_device(c));
  if (c->spectral_order) {
    set_error("the spectral chi0 engine sizes its grid on the host: no graph capture");
    return LRT_EUNSUPPORTED;
  }
  LRT_CUDA(cudaDeviceSynchronize());
  cudaStream_t st = nullptr;
  LRT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  auto done = [&](lrt_status r) {
    cudaStreamDestroy(st);
    return r;
  };
  // an ordinary pass first: plans, buffers, attributes and tuning all settle here
  lrt_status r = forward_all(c, ntau, tau_dev, mode, S_dev, F_dev, metrics_dev, st);
  if (r != LRT_OK) return done(r);
  if (cudaStreamSynchronize(st) != cudaSuccess) return done(LRT_ECUDA);
  r = check_status_word(c);
  if (r != LRT_OK) return done(r);
  const bool prof = c->profiling;
  c->profiling = false;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    c->profiling = prof;
    set_error("stream capture did not start");
    return done(LRT_ECUDA);
  }
  r = forward_all(c, ntau, tau_dev, mode, S_dev, F_dev, metrics_dev, st);
  cudaError_t ee = cudaStreamEndCapture(st, &g);
  c->profiling = prof;
  if (r != LRT_OK || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (r == LRT_OK) {
      set_error(std::string("stream capture: ") + cudaGetErrorString(ee));
      r = LRT_ECUDA;
    }
    return done(r);
  }
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  cudaError_t ie = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    c->graph = nullptr;
    set_error(std::string("graph instantiation: ") + cudaGetErrorString(ie));
    return done(LRT_ECUDA);
  }
  c->graph_valid = true;
  return done(LRT_OK);
}

extern "C" lrt_status lrtddft_graph_launch(lrt_ctx* c, void* stream) {
  if (!c) return bad("NULL context");
  if (!c->graph || !c->graph_valid) {
    set_error("no valid captured graph (capture again after set_params, set_orbitals or set_tuning)");
    return LRT_ESTATE;
  }
  LRT_CUDA(cudaSetDevice(c->device));
  LRT_CUDA(cudaGraphLaunch(c->graph, (cudaStream_t)stream));
  for (auto& Q : c->qd) {
    Q.have_chi0 = Q.have_chi = true;
    Q.have_dchi = false;
  }
  return LRT_OK;
}

extern "C" lrt_status lrtddft_get_pair_densities(lrt_ctx* c, int iq, double* rho) {
  if (!c || !rho) return bad("NULL argument");
  if (iq < 0 || iq >= c->nq) return bad("q index");
  LRT_TRY(need_device(c));
  LRT_TRY(adopt_orbitals(c, iq, 0));
  LRT_CUDA(cudaDeviceSynchronize());
  LRT_TRY(ensure_rho(c));
  const QData& Q = c->qd[iq];
  const bool fp32 = c->precision != LRT_PREC_FP64;
  LRT_TRY(launch_pair_density(c, Q, c->dw.rho, fp32, 0));
  LRT_CUDA(cudaDeviceSynchronize());
  LRT_TRY(check_status_word(c));
  const int nG = Q.nG;
  if (!fp32) {
    std::vector<double2> h((size_t)nG * c->rho_ld);
    LRT_CUDA(cudaMemcpy(h.data(), c->dw.rho, h.size() * sizeof(double2), cudaMemcpyDeviceToHost));
    for (int64_t p = 0; p < c->np; ++p)
      for (int g = 0; g < nG; ++g) {
        rho[2 * (p * nG + g)] = h[(size_t)g * c->rho_ld + p].x;
        rho[2 * (p * nG + g) + 1] = h[(size_t)g * c->rho_ld + p].y;
      }
    return LRT_OK;
  }
  std::vector<float2> h((size_t)c->rho_gpad * c->rho_ld);
  LRT_CUDA(cudaMemcpy(h.data(), c->dw.rho, h.size() * sizeof(float2), cudaMemcpyDeviceToHost));
  const double inv = 1.0 / split_rho_scale(c->precision);
  for (int64_t p = 0; p < c->np; ++p)
    for (int g = 0; g < nG; ++g) {
      const float2 v = h[(((size_t)(p >> 5) * c->rho_gpad + g) << 5) + (size_t)(p & 31)];
      rho[2 * (p * nG + g)] = v.x * inv;
      rho[2 * (p * nG + g) + 1] = v.y * inv;
    }
  return LRT_OK;
}
