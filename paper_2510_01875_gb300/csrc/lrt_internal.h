// Internal declarations of liblrtddft: the context, error plumbing and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lrtddft.h"

namespace lrt {

constexpr double kBasisTol = 1e-9;     // |k+G|^2 <= 2 ecut + kBasisTol
constexpr double kShellTol = 1e-9;     // |q+G|^2 (and |G|^2) closer than this: same shell
constexpr double kPadDiag = 1.0e6;     // Ha; diagonal of the padding rows of H(k)
constexpr double kDegenTol = 1e-6;     // Ha; eigenvalues this close to the last kept band
                                       // form one multiplet (band weights)
constexpr int kExtraBands = 8;         // eigenpairs kept beyond nbands to see such a multiplet

// Thread-local message of the last failure.
void set_error(const std::string& msg);
const char* last_error();

// Tables and buffers of one q on the tensor path, built on first use and kept (they depend on
// the geometry and the frequency list only; weights and sums are refilled per assemble).
struct SplitPlan {
  bool built = false;
  int nsub = 0, n_st = 0, n_n = 0, ldc = 0;   // sub-blocks, row super-tiles, column tiles
  long long ldr = 0;
  size_t pw_n = 0;
  int2* rowtab = nullptr;         // [n_st][8] ring rows of a sub-block's G quads, or (-1, list)
  int2* lsttab = nullptr;         // [n_st][8][16] ring rows of the (G, G') of list slots
  int* blk = nullptr;             // [n_st][6] G blocks per super-tile
  int* rp_of = nullptr;           // [nG][nG] row pair of (G, G')
  float4* wtab = nullptr;         // [n_n][64] frequency pairs (hi, hi, lo, lo)
  float2* etab = nullptr;         // [n_n][64] eta of the two frequencies of each pair
  float4* pw = nullptr;           // [pw_n] (Delta_hi, Delta_lo, df sB, 0)
  double* C = nullptr;            // [ldc][ldr] FP64 sums, column-major
  void* rho = nullptr;            // this q's own pair densities (multi-q launches), or null
};

// Per-q data.  Meshes are indexed s = 0 (k points) and s = 1 (k+q points).
struct QData {
  int nG = 0;
  std::vector<int32_t> gset;      // [nG][3], G = 0 first
  std::vector<double> K;          // [nG]
  std::vector<double> qg2;        // [nG] |q+G|^2
  double* Kdev = nullptr;         // device [nG]
  std::vector<double> kpts;       // [2][nk][3] Cartesian
  std::vector<int32_t> miller;    // [2][nk][npw][3], padding INT32_MIN
  std::vector<int32_t> npw_k;     // [2][nk]
  double mu = 0.0;
  double* eps = nullptr;          // device [2][nk][nb]
  double* occ = nullptr;          // device [2][nk][nb]
  double* wgt = nullptr;          // device [2][nk][nb] band weights (1, 0, or j/m on a split
                                  // degenerate multiplet at the band cut)
  std::vector<double> wgt_h;      // host copy
  double2* coeff = nullptr;       // device [2][nk][nb][npw]
  int32_t* gather = nullptr;      // device [nk][nG][npw]: index into the k+q basis or -1
  double2* chi0 = nullptr;        // device [neta][nwi][nG][nG]
  double2* chi = nullptr;         // device [neta][nwi][nG]  (chi_{G,0})
  bool have_chi0 = false;
  bool have_chi = false;
  std::vector<double> dchi;       // [nwi][5] complex: d chi_00/d(T, eta, A, B, C) (adjoint)
  std::vector<double> ds0;        // [5] complex: d/d(T, eta, A, B, C) of d chi_00/d eta at w = 0
  bool have_dchi = false;
  SplitPlan sp;                   // tensor-path tables of this q
  double sp_x0 = 0.0;             // spectral engine: grid of the last assembly (x_0, bins)
  long long sp_nbins = 0;
  // orbitals of the next assembly, uploaded by lrtddft_set_orbitals_async on the context's
  // upload stream while earlier work runs; swapped with the fields above by adopt_orbitals
  struct Pending {
    bool pending = false;
    double2* coeff = nullptr;     // device [2][nk][nb][npw]
    double* eps = nullptr;        // device [2][nk][nb]
    double* occ = nullptr;
    double* wgt = nullptr;
    std::vector<double> wgt_h;
    double mu = 0.0;
    double* stage = nullptr;      // pinned host [3][2 nk nb]: eps, occ, weights of the copy
    cudaEvent_t ready = nullptr;  // the copies into these buffers have completed
    cudaEvent_t free = nullptr;   // the work that read these buffers (before the swap) is done
  } up;
};

struct DeviceWork {
  void* rho = nullptr;            // FP64 path: [nGmax][rho_ld] complex; split path: FP32
                                  // complex blocked [rho_ld / 32][rho_gpad][32]
  size_t rho_bytes = 0;
  double* delta = nullptr;        // [np]
  double* df = nullptr;           // [np]
  double* freqs = nullptr;        // [nwi]
  double* omega = nullptr;        // [nw]
  double* S = nullptr;            // [nq][neta][nw]
  double* chi00 = nullptr;        // [nq][neta][nwi][2] gather of chi_00 for the spectra kernels
  int* status = nullptr;          // device status word (0 ok, bit 1 singular, bit 2 timeout)
  double* scratch = nullptr;      // tensor path: FP64 sums of the contraction
  size_t scratch_bytes = 0;
  void* pd_work = nullptr;        // tensor-core pair densities: prepared operands of one q
  size_t pd_bytes = 0;
  double* zt_part = nullptr;      // tensor-core w = 0 column: per-CTA FP64 partial sums
  size_t zt_bytes = 0;
  void* dyson_ws = nullptr;       // Dyson matrices of N_G too large for shared memory
  size_t dyson_bytes = 0;
  double2* s0 = nullptr;          // [nq][neta] d chi_00/d eta at w = 0 (S(q,0) = T Re s0/(pi n))
  int* eta_ref = nullptr;         // [nq] reference eta of the last eta scan
  double2* zf = nullptr;          // zero-frequency vectors: x, u, v and the adjoint's pieces
  void* zf_ws = nullptr;          // matrix of the zero-frequency LU when it exceeds shared memory
  size_t zf_ws_bytes = 0;
};

}  // namespace lrt

struct lrt_ctx {
  // inputs
  double lattice[3][3];
  double recip[3][3];
  double volume = 0.0;
  std::vector<double> positions;  // [natoms][3]
  int natoms = 0;
  double Z = 0.0, r_c = 0.0, ecut = 0.0;
  int potential = 0, basis = 0;
  int kn[3] = {1, 1, 1};
  int kscheme = 0;
  int nk = 0;
  int nbands = 0;                 // bands requested per k point
  int nb = 0;                     // bands carried: nbands plus split-multiplet members
  double T = 0.0, eta = 0.0;      // eta: the broadening (the smallest of the eta list)
  int neta = 1;                   // broadenings per context (lrtddft_set_eta_list)
  std::vector<double> etas;       // [neta] ascending; {eta} unless a list was set
  int nq = 0;
  std::vector<double> q;          // [nq][3]
  int nw = 0;
  std::vector<double> omega;      // [nw]
  std::vector<double> freqs;      // [nwi] internal frequencies
  int nwi = 0;
  int hcol = 0;
  lrt_kernel kernel{};
  int precision = 0;
  int device = 0;
  double density = 0.0;           // N_e / Omega
  double nelec = 0.0;
  double fxc = 0.0;               // f_ALDA at the mean density
  int npw = 0;                    // padded plane-wave count (max over all k points)
  int nGmax = 0;
  int64_t np = 0;                 // pairs per q = nk nb^2
  int64_t rho_ld = 0;             // np rounded up to 32 (whole 32-pair stages)
  int rho_gpad = 0;               // split path: G count padded to 8 of the blocked rho layout
  std::vector<lrt::QData> qd;
  lrt::DeviceWork dw;
  bool have_S = false;
  bool host_only = false;
  // instrumentation (lrtddft_profile): launch counter and event pairs around the chi0
  // contraction and pair-density launches
  mutable long long launches = 0;
  bool profiling = false;
  mutable std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_chi0, ev_rho;
  mutable double timed_cmac = 0.0;
  // tensor path: launch state, tuning (lrtddft_set_tuning) and the last choice made
  void* tc = nullptr;
  bool autotune = false;
  bool multi_q = true;
  bool pair_simt = false;         // split-path pair densities on the FP32 SIMT kernel
  bool fine_accum = false;        // FP32 accumulation period of 32 stages instead of 64
  bool half_tiles = false;        // forced half row units (256 rows per CTA pair)
  bool zero_simt = false;         // split w = 0 column on the CUDA cores, not the tensor cores
  int spectral_order = 0;         // chi0 engine: 0 the direct pair sum, 1 or 3 the spectral
  double spectral_h = 0.0;        // function on a grid of this spacing (interpolation order)
  void* sp = nullptr;             // spectral engine state (spectral.cu)
  int last_tc_rows = 0;           // rows per CTA-pair unit of the last tensor launch (512, 256)
  int tune_variant = -1;          // forced kernel variant, -1: tuned or default
  int tune_unit_stages = 0;       // forced stages per unit, 0: tuned or default
  int last_tc_variant = -1, last_tc_unit_stages = 0;
  // Kubo-Greenwood scan (kubo.cu): S*_KG rows and the reference eta of the last scan
  void* kg = nullptr;
  // captured forward graph (lrtddft_graph_capture)
  cudaStream_t upload = nullptr;    // lrtddft_set_orbitals_async copies (non-blocking stream)
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
};

namespace lrt {
// Columns of chi0 per q (every internal frequency for every eta, eta-major) and rows of the
// spectra (S, F, metrics: every q for every eta, q-major).
inline int ncol(const lrt_ctx* c) { return c->neta * c->nwi; }
inline int nrow(const lrt_ctx* c) { return c->nq * c->neta; }
// Count kernel launches for lrtddft_profile_read.
inline void count_launch(const lrt_ctx* c, int n = 1) { c->launches += n; }
inline cudaEvent_t new_event();
// With profiling on, record an event pair around one launch: begin() before, end() after.
struct TimedLaunch {
  const lrt_ctx* c;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* list;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  TimedLaunch(const lrt_ctx* ctx, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* l,
              cudaStream_t st)
      : c(ctx), list(l), s(st) {
    if (c->profiling) {
      a = new_event();
      cudaEventRecord(a, s);
    }
  }
  ~TimedLaunch() {
    if (c->profiling) {
      cudaEvent_t b = new_event();
      cudaEventRecord(b, s);
      list->emplace_back(a, b);
    }
  }
};
inline cudaEvent_t new_event() {
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace lrt

namespace lrt {

// setup.cu
lrt_status build_geometry(lrt_ctx* c, const int* nG);
lrt_status solve_ground_states(lrt_ctx* c, const double* occupations);
lrt_status set_occupations_fd(lrt_ctx* c, int iq, const double* eps_host);
lrt_status reset_band_weights(lrt_ctx* c, int iq, const double* eps_host);
lrt_status fermi_occupations(const lrt_ctx* c, const double* eps_host, const double* wgt,
                             double* f, double* mu);
lrt_status band_weights_all(const lrt_ctx* c, const double* eps_host, double* out);
lrt_status adopt_orbitals(lrt_ctx* c, int iq, cudaStream_t s);
lrt_status launch_chi0_spectral(lrt_ctx* c, QData& q, const void* rho, cudaStream_t s);
void free_spectral_state(lrt_ctx* c);
lrt_status split_pair_weights(const lrt_ctx* c, QData& q, float* sB, cudaStream_t s);
lrt_status launch_zero_split(const lrt_ctx* c, QData& q, const void* rho, float sB, cudaStream_t s);
// zero_tc.cu: the same column on the tensor cores (*done false when it does not apply)
lrt_status launch_zero_tc(const lrt_ctx* c, QData& q, const void* rho, float sB, cudaStream_t s,
                          bool* done);
double fxc_alda(double n);
double fxc_model(double qg, double n, double A, double B, double C);
// K_GG = 4 pi/|q+G|^2 + f_xc for the context's kernel, from Q.qg2 (host vector only).
void kernel_diag(const lrt_ctx* c, QData& Q);

// Power-of-two factor carried by the FP32 pair densities of the split-precision path (FP16
// parts: keeps the products rho rho* clear of the FP16 subnormal range; exact in binary).
inline float split_rho_scale(int precision) { return precision == LRT_PREC_FP16X3 ? 128.0f : 1.0f; }

// pairdens.cu: rho[G][p] for one q (FP64 or FP32 storage)
lrt_status launch_pair_density(const lrt_ctx* c, const QData& q, void* rho, bool fp32,
                               cudaStream_t s);
lrt_status launch_pair_weights(const lrt_ctx* c, const QData& q, cudaStream_t s);
// pairdens_tc.cu: split-path (blocked FP32) pair densities on the tensor cores
lrt_status launch_pair_density_tc(const lrt_ctx* c, const QData& q, void* rho, cudaStream_t s);

// chi0_fp64.cu
lrt_status launch_chi0_fp64(const lrt_ctx* c, QData& q, cudaStream_t s);
// chi0_tc.cu: chi0 of q_begin .. q_end - 1 on the tensor path (one launch for all q whose
// pair densities fit in their own buffers)
lrt_status launch_chi0_split_range(lrt_ctx* c, int q_begin, int q_end, cudaStream_t s);
void free_split_plan(SplitPlan& sp);
void free_tc_state(lrt_ctx* c);
// api.cu: the shared pair-density buffer; the device status word (timeout before singular)
lrt_status ensure_rho(lrt_ctx* c);
lrt_status check_status_word(const lrt_ctx* c);

// dyson.cu
lrt_status launch_dyson(const lrt_ctx* c, QData& q, int iq, cudaStream_t s);

// zerofreq.cu: the w -> 0 limit of Eq. 8, S(q,0) = (T/(pi n)) Re d chi_00/d eta at w = 0
lrt_status ensure_zf(lrt_ctx* c);
lrt_status launch_lu_two_solves(const lrt_ctx* c, const QData& q, int w, const double2* rhs_n,
                                const double2* rhs_t, const double* tscale, double2* out_n,
                                double2* out_t, double2* v_out, cudaStream_t s);
lrt_status launch_s0(const lrt_ctx* c, const QData& q, int iq, const void* rho, const float4* pw,
                     float sB, cudaStream_t s);
lrt_status launch_s0_tangents(const lrt_ctx* c, const QData& q, const double2* u, const double2* v,
                              const double* d_dK, const double* delta, const double* df,
                              const double* ddf, double* ds_host, cudaStream_t s);

// spectra.cu
lrt_status launch_dsf(const lrt_ctx* c, double* S_dev, cudaStream_t s);
lrt_status launch_itcf(const lrt_ctx* c, const double* S_dev, int ntau, const double* tau_dev,
                       int mode, double* F_dev, double* metrics_dev, cudaStream_t s);
// the same on explicit rows of S [rows][nw] with their S(0) values s0 [rows] (S(0) = T Re s0/(pi n))
lrt_status launch_itcf_rows(const lrt_ctx* c, const double* S_dev, const double2* s0_dev, int rows,
                            int ntau, const double* tau_dev, int mode, double* F_dev,
                            double* metrics_dev, cudaStream_t s);
// reference eta per q from metrics [nq][neta][5] (Sec. 2)
lrt_status launch_eta_pick(const lrt_ctx* c, const double* metrics_dev, int nq, int neta, double tol,
                           int* ref_dev, cudaStream_t s);

// adjoint.cu: d chi_00/d(T, eta, A, B, C) at every internal frequency of one q, out[nwi][10]
// (complex pairs); needs the q's chi0, chi and pair densities (in dw.rho)
lrt_status launch_adjoint_q(const lrt_ctx* c, QData& q, int iq, std::vector<double>& out,
                            cudaStream_t s);

// attenuate.cu: the context's spectrum rows, or explicit rows S [rows][nw] with s0 [rows]
lrt_status run_attenuation(const lrt_ctx* c, const lrt_atten_params* p, const double* S_dev,
                           double* Sp_host, lrt_atten_report* rep, cudaStream_t s);
lrt_status run_attenuation_rows(const lrt_ctx* c, const lrt_atten_params* p, const double* S_dev,
                                const double2* s0_dev, int rows, double* Sp_host,
                                lrt_atten_report* rep, cudaStream_t s);

// kubo.cu
void free_kg_state(lrt_ctx* c);

// dielectric.cu: Kramers-Kronig and Eqs. 10-11 on rows S [rows][nw] (host), v [rows] the
// Coulomb factor per row; out [rows][N][8] (host)
lrt_status run_dielectric(const lrt_ctx* c, const double* S_host, int rows, const double* v,
                          double* out_host);

}  // namespace lrt

#define LRT_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      lrt::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));               \
      return (e_ == cudaErrorMemoryAllocation) ? LRT_ENOMEM : LRT_ECUDA;                \
    }                                                                                   \
  } while (0)

#define LRT_TRY(call)                                                                   \
  do {                                                                                  \
    lrt_status s_ = (call);                                                             \
    if (s_ != LRT_OK) return s_;                                                        \
  } while (0)
