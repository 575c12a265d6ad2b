/*
 * lrtddft.h -- C ABI of the GB300 linear-response TDDFT response library (liblrtddft.so).
 *
 * The library computes, for a list of momentum transfers q, the dynamic structure factor
 * S(q,w) and the imaginary-time correlation function F(q,tau) of a crystal with a fixed
 * (non-self-consistent) empty-core pseudopotential, and the constraints-based attenuation
 * of narrow-band fluctuations of S:
 *
 *   rho_p(G)      = <nk| e^{-i(q+G).r} |n'k+q>,  p = (k, n, n')            (pair densities)
 *   chi0_GG'(q,w) = (2/(N_k Omega)) sum_p rho_p(G) rho_p*(G') (f_nk - f_n'k+q)
 *                                              / (w + eps_nk - eps_n'k+q + i eta)
 *                                                        (Adler-Wiser independent-particle)
 *   chi           = (1 - chi0 K)^{-1} chi0,  K_GG' = delta_GG' (4 pi/|q+G|^2 + f_xc)  (Dyson)
 *   S(q,w)        = -Im chi_00(q,w) / (pi n (1 - e^{-w/T}))   fluctuation-dissipation, Eq. 8
 *   F(q,tau)      = int dw S(q,w) e^{-tau w}, with S(q,-w) = e^{-w/T} S(q,w)
 *                                           two-sided Laplace transform + detailed balance, Eq. 1
 *   F~(q,tau)     = F(q,tau) - F(q,0)                                                   Eq. 2
 *   attenuation   Savitzky-Golay grid search scored by AICc + penalties, accepted under the
 *                 imaginary-time constraints of Sec. 3, Eqs. 5-7.
 * (Section, equation numbers: Moldabekov et al., "Enhancing the Efficiency of TDDFT
 * Calculations of Dynamic Response Properties".  The chi0/Dyson engine itself is the
 * textbook Adler-Wiser + Dyson form; the paper's own engine is Liouville-Lanczos.)
 *
 * Conventions for every entry point:
 *  - Units: Hartree atomic units (Ha, bohr, 1/bohr); temperature T in Ha.
 *  - Arrays are row-major, C order, with the sizes given in each comment.  Complex numbers
 *    are (re, im) pairs of doubles.
 *  - Ownership: inputs are read during the call and copied; the caller keeps them.  Outputs
 *    go to caller-owned buffers.  Functions named *_device take device pointers and a
 *    cudaStream_t (passed as void*) and return once the work is enqueued; the others take
 *    host pointers and return after the results are on the host.  The library owns all of
 *    its device workspace and frees it in lrtddft_destroy.
 *  - Errors: every function returns an lrt_status; nothing throws or aborts across the ABI.
 *    lrtddft_status_string gives a message and lrtddft_last_error the detail of the last
 *    failure on the calling thread.  After LRT_ECUDA the context must be destroyed.
 *  - One context is used from one host thread at a time.
 */
#ifndef LRTDDFT_H
#define LRTDDFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LRT_OK = 0,
  LRT_EINVAL = 1,       /* invalid argument (sizes, grids, q equal to a lattice vector ...) */
  LRT_ENOMEM = 2,       /* device or host allocation failed */
  LRT_ECUDA = 3,        /* CUDA / cuSOLVER error */
  LRT_ESINGULAR = 4,    /* a Dyson matrix 1 - chi0 K had a zero pivot */
  LRT_ETIMEOUT = 5,     /* a bounded device-side wait ran out */
  LRT_ESTATE = 6,       /* calls out of order (e.g. dsf before dyson_solve) */
  LRT_EUNSUPPORTED = 7  /* option not available in this build / on this device */
} lrt_status;

typedef struct lrt_ctx lrt_ctx;

enum { LRT_POT_EMPTY_CORE = 0, LRT_POT_ZERO = 1 };
enum { LRT_BASIS_SPHERE = 0, LRT_BASIS_FIXED = 1 };
enum { LRT_K_COMMENSURATE = 0, LRT_K_TR_SYMMETRIC = 1 };
enum { LRT_KERNEL_RPA = 0, LRT_KERNEL_RPA_ALDA = 1, LRT_KERNEL_FXC_MODEL = 2 };
/* Precision of the pair densities and the chi0 contraction (the Dyson solve, S and F are
 * always FP64):
 * FP64: FP64 products and sums;  FP16X3 / BF16X3: pair densities in FP32 (tensor cores with a
 * fixed-grid FP16 split whose high products are summed exactly, 128-band blocks), and each
 * contraction operand split into a high and a low 16-bit part, three
 * tensor-core products (hi*hi + hi*lo + lo*hi) accumulated in FP32 and flushed into FP64
 * partial sums.  FP16X3 is the FP32-emulating form (hi + lo carry about 22 bits). */
enum { LRT_PREC_FP64 = 0, LRT_PREC_FP16X3 = 1, LRT_PREC_BF16X3 = 2 };
enum { LRT_ITCF_FOLD = 0, LRT_ITCF_DIRECT = 1 };

/* Crystal and plane-wave basis.  V(G) = sum_a v(|G|) e^{-i G.R_a},
 * v(G) = -(4 pi Z/(Omega G^2)) cos(G r_c) (Ashcroft empty core), V(0) = 0.
 * Basis per k: {G : |k+G|^2/2 <= ecut} (SPHERE) or {G : |G|^2/2 <= ecut} (FIXED). */
typedef struct {
  double lattice[3][3];     /* rows are the lattice vectors, bohr */
  int natoms;
  const double* positions;  /* [natoms][3] Cartesian, bohr */
  double Z;                 /* ionic valence; N_e = Z * natoms */
  double r_c;               /* empty-core radius, bohr */
  double ecut;              /* Ha */
  int potential;            /* LRT_POT_* */
  int basis;                /* LRT_BASIS_* */
} lrt_cell;

/* k-mesh: Gamma-centred M = {sum_j (i_j/n_j) b_j}.  COMMENSURATE: k in M, k+q = k + q.
 * TR_SYMMETRIC: k in M - q/2, k+q in M + q/2 (then -k-q lies in the k set modulo G, so
 * chi0(-w)* = chi0(w)^T and detailed balance holds to rounding). */
typedef struct {
  int n[3];
  int scheme;               /* LRT_K_* */
} lrt_kmesh;

/* Static kernel added to the Coulomb term: RPA (none), RPA_ALDA (f_xc of the mean density:
 * Slater exchange + Perdew-Wang 1992 correlation), FXC_MODEL:
 * f_xc(|q+G|) = A f_ALDA (1 + B |q+G|^2) exp(-C |q+G|^2). */
typedef struct {
  int kind;                 /* LRT_KERNEL_* */
  double A, B, C;
} lrt_kernel;

/* flags: LRT_FLAG_HOST_ONLY builds only the host-side geometry (k meshes, bases, G-sets,
 * K) and touches no GPU; compute calls on such a context return LRT_ESTATE. */
enum { LRT_FLAG_HOST_ONLY = 1 };
typedef struct {
  int precision;            /* LRT_PREC_* */
  int device;               /* CUDA device ordinal */
  int flags;                /* LRT_FLAG_* */
} lrt_options;

/* Create a context: builds the k meshes, bases and response G-sets, diagonalises H(k) on
 * the GPU (cuSOLVER, setup only), sets occupations and the Dyson kernel.
 *   nbands        bands kept per k point (<= plane waves at every k)
 *   T             electron temperature, Ha (> 0)
 *   occupations   NULL for Fermi-Dirac with mu from (2/N_k) sum f = N_e on the k mesh of each
 *                 q; else [nq][2][nk][nbands] (k mesh, then k+q mesh) overriding f
 *   q             [nq][3] Cartesian, 1/bohr; no q may be a reciprocal-lattice vector
 *   nG            [nq] response G-vectors per q: the nG of smallest |q+G| (ties: smaller |G|,
 *                 then lexicographic Miller indices), ordered with G = 0 first
 *   omega         [nw] strictly increasing real frequencies, Ha
 *   eta           Lorentzian broadening, Ha (> 0)
 * Errors: EINVAL (sizes, non-monotone omega, nbands too large, G = 0 not in the set),
 * ENOMEM, ECUDA. */
lrt_status lrtddft_create(const lrt_cell* cell, const lrt_kmesh* kmesh, int nbands, double T,
                          const double* occupations, int nq, const double* q, const int* nG,
                          int nw, const double* omega, double eta, const lrt_kernel* kernel,
                          const lrt_options* opt, lrt_ctx** out);

lrt_status lrtddft_destroy(lrt_ctx* ctx);

const char* lrtddft_status_string(lrt_status s);
/* Detail of the last failure on this thread (static storage; valid until the next call). */
const char* lrtddft_last_error(void);

/* Sizes of a context: out[0..7] = nq, nw, nk, nb (bands carried per k point: nbands plus the
 * members of any degenerate multiplet split by the band cut), max nG, plane waves (padded), number of
 * internal frequencies (nw plus a w = 0 column when 0 is not on the grid), precision. */
lrt_status lrtddft_query(const lrt_ctx* ctx, int64_t out[8]);

/* chi0 for q in [q_begin, q_end): pair densities (G-space correlation of the orbitals) and
 * the Adler-Wiser contraction at every internal frequency, kept on the device, and
 * d chi_00/d eta at w = 0 (for S(q,0)).  Enqueued on `stream` (cudaStream_t; NULL = legacy
 * default stream). */
lrt_status lrtddft_chi0_assemble(lrt_ctx* ctx, int q_begin, int q_end, void* stream);

/* Dyson for q in [q_begin, q_end): solves (1 - chi0 K) x = chi0_{:,0} by LU with partial
 * pivoting per (q, w), FP64; x = chi_{G,0}.  Requires chi0_assemble on the same q.
 * A zero pivot makes a later synchronising call return LRT_ESINGULAR. */
lrt_status lrtddft_dyson_solve(lrt_ctx* ctx, int q_begin, int q_end, void* stream);

/* S(q,w) (Eq. 8) on the caller's grid: S [nq][nw].  At w = 0 the exact limit of Eq. 8 is
 * used: S(q,0) = -(T/(pi n)) d Im chi_00/dw = (T/(pi n)) Re d chi_00/d eta at w = 0 (chi_00 is
 * analytic in w + i eta), with d chi_00/d eta from the Dyson chain rule and a projection of
 * the pair densities computed by chi0_assemble.  Requires dyson_solve for every q. */
lrt_status lrtddft_dsf(lrt_ctx* ctx, double* S);
lrt_status lrtddft_dsf_device(lrt_ctx* ctx, double* S_dev, void* stream);

/* F(q,tau) at the caller's tau (each in [0, 1/T]):
 *   FOLD   (Eq. 1 with detailed balance) trapezoid over the w >= 0 samples (plus w = 0) of
 *          S(w)[e^{-tau w} + e^{-(1/T - tau) w}];
 *   DIRECT trapezoid over the whole caller grid of S(w) e^{-tau w}.
 * F [nq][ntau]; metrics [nq][5] (may be NULL) = F(beta/2), int_0^beta F dtau,
 * F~(beta/2) (Eq. 2), int_0^beta F~ dtau and the static response -n int_0^beta F dtau
 * (Sec. 2), the tau integrals done exactly per w (FOLD branch). */
lrt_status lrtddft_itcf_laplace(lrt_ctx* ctx, int ntau, const double* tau, int mode, double* F,
                                double* metrics);
lrt_status lrtddft_itcf_laplace_device(lrt_ctx* ctx, int ntau, const double* tau_dev, int mode,
                                       double* F_dev, double* metrics_dev, void* stream);

/* ---- Scheduling of the tensor-core contraction (FP16X3 / BF16X3; no effect on FP64).
 * chi0_assemble runs all requested q in one persistent launch when their pair densities fit
 * next to each other in device memory (q of different N_G mix freely: the launch walks a list
 * of (q, row unit, column tile, pair range) units); otherwise q by q.  A row unit is 512 rows
 * of the Hermitian-split chi0 (256 per CTA of the pair, two accumulators each) or, as a half,
 * 256 rows (128 per CTA); an odd last unit is always a half.  Each unit covers a fixed number
 * of 32-pair stages ("unit size"), and two kernel variants differ in their shared-memory ring
 * depths (0: 4 operand / 2 prefetch stages, 1: 3 / 4).
 *   flags: LRT_TUNE_AUTO      time each (row unit shape, variant, unit size) candidate on the
 *                             first units of the first launch of each shape and keep the
 *                             fastest (results then differ from the defaults at the rounding
 *                             of the split form);
 *          LRT_TUNE_SINGLE_Q  one launch per q;
 *          LRT_TUNE_PAIR_SIMT pair densities on the FP32 SIMT kernel instead of the tensor
 *                             cores;
 *          LRT_TUNE_FINE_ACCUM flush the FP32 tensor-core accumulators into the FP64 sums every
 *                             32 stages (1024 pairs) instead of 64: the FP32 accumulation
 *                             error, which grows with the period, halves;
 *          LRT_TUNE_HALF_TILES every row unit a half (256 rows; more, smaller units);
 *          LRT_TUNE_ZERO_SIMT  the split forms' w = 0 column (when 0 is not on the grid) on
 *                             the CUDA cores instead of the tensor cores (the tensor-core
 *                             kernel takes 64 x 64 G tiles, at least one SM each: with more
 *                             tiles than SMs, N_G > 768 on 152 SMs, the CUDA-core kernel runs
 *                             in any case).
 *   variant: -1 (tuned or default 0), 0 or 1;  unit_stages: 0 (tuned or default 4096) or a
 *   positive multiple of 64.  LRT_EINVAL otherwise.  Invalidates a captured graph. */
enum { LRT_TUNE_AUTO = 1, LRT_TUNE_SINGLE_Q = 2, LRT_TUNE_PAIR_SIMT = 4, LRT_TUNE_FINE_ACCUM = 8,
       LRT_TUNE_HALF_TILES = 16, LRT_TUNE_ZERO_SIMT = 32 };
lrt_status lrtddft_set_tuning(lrt_ctx* ctx, int flags, int variant, int unit_stages);
/* The variant and unit size used by the last tensor-core launch (-1 and 0 before any). */
lrt_status lrtddft_get_tuning(lrt_ctx* ctx, int* variant, int* unit_stages);
/* Rows of chi0 per full row unit of the last tensor-core launch: 512, or 256 when every unit
 * was a half (0 before any). */
lrt_status lrtddft_get_tile_rows(lrt_ctx* ctx, int* rows);

/* ---- chi0 through a spectral function (an engine variant; the paper's method is the direct
 * Adler-Wiser sum above).  With x_p = eps_n'k+q - eps_nk, every pole 1/(w - x_p + i eta) of
 * the sum is replaced by its Lagrange interpolant of order `order` (1 or 3) in x_p on the grid
 * x_b = x_0 + b h: A_b(G,G') = sum_p rho_p(G) rho_p*(G') df_p L_b(x_p) is formed once from the
 * pairs sorted by bin, and chi0(w) = (2/(N_k Omega)) sum_b A_b / (w - x_b + i eta) for every
 * frequency and every eta of a list is one GEMM over the bins.  The relative error is
 * O((h/eta)^(order+1)) (order 3, h = eta/16: about 1e-6 of max |chi0|); the cost of the pair
 * sum no longer grows with the number of frequencies.  Grid: over the pairs with df != 0,
 * x_0 = h (floor(min x_p / h) - 1), n_b = floor((max x_p - x_0)/h) + 3.  The FP64 context forms
 * A in FP64 and transforms with cuBLAS DGEMM; the split contexts form A from FP32 products with
 * compensated FP32 sums per bin and transform with FP32 products accumulated over 256 bins at
 * a time (cuBLAS SGEMM, strided batches), the chunks summed in FP64.  S(q,0) keeps its exact
 * limit.  h = 0 selects the direct engine
 * (the default).  Not with the adjoint or graph capture (LRT_EUNSUPPORTED there).  LRT_EINVAL
 * for h < 0 or an order other than 1, 3; chi0_assemble returns LRT_EINVAL when the grid would
 * exceed 2^26 bins. */
lrt_status lrtddft_set_spectral(lrt_ctx* ctx, double h, int order);
/* Grid of the last spectral assembly of q index iq: x_0 (Ha) and the number of bins (0 and 0
 * before one, or when no pair carries weight). */
lrt_status lrtddft_get_spectral_grid(const lrt_ctx* ctx, int iq, double* x0, long long* nbins);

/* CUDA graph of the forward path for every q: chi0_assemble, dyson_solve, dsf_device and
 * itcf_laplace_device into the given device buffers (S_dev [nq][nw], F_dev [nq][ntau],
 * metrics_dev [nq][5], tau_dev [ntau]; they must stay allocated).  One ordinary pass runs
 * first (it builds the tables, allocates, tunes), then the same calls are captured on a
 * private stream and instantiated.  graph_launch replays it on `stream`; it returns
 * LRT_ESTATE when there is no graph or after set_params, set_orbitals or set_tuning (capture
 * again).  Attenuation is not part of the graph (its candidate search runs on the host). */
lrt_status lrtddft_graph_capture(lrt_ctx* ctx, int ntau, const double* tau_dev, int mode,
                                 double* S_dev, double* F_dev, double* metrics_dev);
lrt_status lrtddft_graph_launch(lrt_ctx* ctx, void* stream);

/* ---- The eta-convergence test in the imaginary-time domain (Sec. 2, Eqs. 1-2).
 * An eta list makes every later chi0_assemble compute chi0 for all of its broadenings from one
 * pass of pair densities: the tensor-core contraction takes the (eta, w) pairs as the columns
 * of one launch (the FP64 form runs one contraction per eta); dyson_solve then solves every
 * (eta, w), and S, F and the metrics come as rows (q, eta), q-major:
 *   dsf S [nq][n_eta][nw],  itcf_laplace F [nq][n_eta][ntau], metrics [nq][n_eta][5],
 *   attenuate S_p [nq][n_eta][nw] and report [nq][n_eta],
 *   get_chi0 [n_eta][nw_int][nG][nG],  get_chi_col0 [n_eta][nw_int][nG]
 * (with one eta these are the shapes given elsewhere).  The adjoint calls (jacobian, the vjps)
 * take a single eta and return LRT_EUNSUPPORTED otherwise; set_params returns to the single
 * eta it is given. */

/* eta [n_eta] strictly increasing broadenings, Ha (> 0), 1 <= n_eta <= 64.  Drops chi0 and chi
 * (chi0_assemble and dyson_solve must run again) and invalidates a captured graph.  LRT_EINVAL
 * for a bad list. */
lrt_status lrtddft_set_eta_list(lrt_ctx* ctx, int n_eta, const double* eta);
/* The current list: *n_eta and, if eta is not NULL, eta [n_eta]. */
lrt_status lrtddft_get_eta_list(const lrt_ctx* ctx, int* n_eta, double* eta);
/* The convergence test after dyson_solve on every q: F (FOLD form of Eq. 1) at the caller's
 * tau and the metrics of itcf_laplace for every (q, eta) (F and metrics may be NULL), and
 * eta_ref [nq], the index of each q's reference eta: the largest eta_j of the converged range,
 * read as: for every i <= j both F~(beta/2) and int_0^beta F~ (Eq. 2) lie within
 * tol |m(eta_0)| of their value m(eta_0) at the smallest eta (the paper's criterion, Sec. 2, is
 * qualitative; tol sets it).  Host buffers. */
lrt_status lrtddft_eta_scan(lrt_ctx* ctx, int ntau, const double* tau, double tol, double* F,
                            double* metrics, int* eta_ref);

/* ---- Dielectric properties from a DSF (Sec. 3, closing relations; App. A.2, Eqs. 10-11).
 * From S (typically the S_p of lrtddft_attenuate) on the context's grid, rows as lrtddft_dsf
 * returns them ([nq][n_eta][nw]), at the N samples with w >= 0 (uniformly spaced, N >= 3):
 *   Im chi = -pi n (1 - e^{-w/T}) S  (Eq. 8),
 *   Re chi = (2/pi) P int_0^inf w' Im chi(w')/(w'^2 - w^2) dw'  (Kramers-Kronig; the principal
 *            value by Maclaurin's formula on the samples, Ohta and Ishida 1988, second order in
 *            the spacing, the range below the first and above the last sample left out),
 *   1/eps = 1 + (4 pi/|q|^2) chi  (Eq. 10),  eps,  sigma = (i w/(4 pi)) (1 - eps)  (Eq. 11).
 * out [rows][N][8] = Re chi, Im chi, Re 1/eps, Im 1/eps, Re eps, Im eps, Re sigma, Im sigma.
 * Host buffers.  LRT_EINVAL for a grid without 3 uniformly spaced samples w >= 0. */
lrt_status lrtddft_dielectric(lrt_ctx* ctx, const double* S, double* out);

/* ---- Parameters and adjoint.  theta = (T, eta, A, B, C): temperature, broadening and the
 * three parameters of the FXC_MODEL kernel (for RPA and RPA_ALDA the A, B, C components are
 * 0).  The paper fits none of these by gradients; these calls serve fitting T and kernel
 * parameters to measured spectra through the same response path (S by Eq. 8, F by the
 * detailed-balance fold of Eq. 1). */

/* New T (Ha), eta (Ha) and kernel for an existing context, without new eigensolves (the
 * orbitals do not depend on them here): Fermi-Dirac occupations and mu are recomputed at T
 * (occupations supplied by the caller stay as they are), K is rebuilt, and chi0, chi and the
 * derivatives are invalidated, so chi0_assemble and dyson_solve must run again.
 * LRT_EINVAL for T <= 0, eta <= 0, an unknown kernel kind or non-finite A, B, C. */
lrt_status lrtddft_set_params(lrt_ctx* ctx, double T, double eta, const lrt_kernel* kernel);

/* Derivatives with respect to theta at the current state (requires dyson_solve for every q):
 *   dS [nq][nw][5]    dS(q, w)/dtheta on the caller's grid (NULL to skip);
 *   dF [nq][ntau][5]  dF(q, tau)/dtheta of the FOLD form at the absolute times tau[ntau]
 *                     (held fixed when T changes; NULL to skip, then tau may be NULL).
 * The first call after chi0/chi changed recomputes the pair densities of every q, the Dyson
 * LU from the stored chi0 (M^T u = e_0, M = 1 - chi0 K), and the projections
 * sum_p (u.rho_p)(rho_p^*.v) dw_p/dtheta (2 N_G complex MACs per pair and frequency) on the
 * GPU; the results are kept until chi0, chi or the parameters change.  Errors as
 * itcf_laplace; LRT_ESINGULAR if a Dyson matrix is singular. */
lrt_status lrtddft_jacobian(lrt_ctx* ctx, int ntau, const double* tau, double* dS, double* dF);

/* Vector-Jacobian products: grad[5] = sum_{q,tau} dL_dF[q][tau] dF(q,tau)/dtheta (FOLD form,
 * absolute tau[ntau] as in itcf_laplace) and grad[5] = sum_{q,w} dL_dS[q][w] dS(q,w)/dtheta.
 * Host buffers; same requirements and caching as lrtddft_jacobian. */
lrt_status lrtddft_itcf_vjp(lrt_ctx* ctx, int ntau, const double* tau, const double* dL_dF,
                            double grad[5]);
lrt_status lrtddft_dsf_vjp(lrt_ctx* ctx, const double* dL_dS, double grad[5]);

/* Attenuation of narrow-band fluctuations (Sec. 3).  Defaults (fields <= 0) in brackets. */
typedef struct {
  int d_min, d_max;         /* polynomial degrees searched [1, 4] */
  double w_min, w_max;      /* window grid, Ha, full widths [4 dw, quarter of the range] */
  int n_w;                  /* windows in the grid [24]; m = 2 round(w/(2 dw)) + 1 points */
  double lambda_f;          /* weight of ln(max(R_f, r0)/r0), R_f = target power kept [N] */
  double lambda_c;          /* weight of the second-difference ratio [N] */
  int n_targets;            /* strongest local maxima of the dS/dw periodogram [2] */
  double feat_lo, feat_hi;  /* featureless range, Ha [central 90 % of the w >= 0 samples] */
  double low_exclude;       /* lowest fraction of Fourier frequencies ignored [0.05] */
  double accept_mean;       /* |Fbar_n| / F(beta/2) limit [4e-3] (Sec. 3) */
  double accept_rms;        /* sigma_n / F(beta/2) limit [4.2e-5] (Sec. 3) */
  int average;              /* 0 or 1: S_p = mean over the accepted degrees (Sec. 4.1);
                               2: the accepted degree with the lowest score */
  int ntau;                 /* tau points on [0, beta/2] for the constraints [64] */
  double retain_floor;      /* r0 [1e-4] */
} lrt_atten_params;

#define LRT_ATTEN_MAX_DEG 8
typedef struct {
  int n_accepted;
  int targets[4];           /* periodogram bins of the targets (-1 = none) */
  int degree[LRT_ATTEN_MAX_DEG];       /* degree d of each row (-1 = unused) */
  int window[LRT_ATTEN_MAX_DEG];       /* chosen window m (points) */
  double score[LRT_ATTEN_MAX_DEG];
  double mean_ratio[LRT_ATTEN_MAX_DEG];  /* |Fbar_n| / F(beta/2) */
  double rms_ratio[LRT_ATTEN_MAX_DEG];   /* sigma_n / F(beta/2) */
  int accepted[LRT_ATTEN_MAX_DEG];
} lrt_atten_report;

/* Sp [nq][nw] (samples with w < 0 are copied from S unchanged); report [nq] (may be NULL).
 * Requires dyson_solve for every q and at least 8 uniformly spaced samples with w >= 0. */
lrt_status lrtddft_attenuate(lrt_ctx* ctx, const lrt_atten_params* params, double* Sp,
                             lrt_atten_report* report);

/* Allocation-free lrtddft_attenuate: same arguments, results and errors, but no device memory
 * is allocated during the call.  The paper has no counterpart; this exists for callers that
 * cannot call cudaMalloc/cudaFree when they attenuate: programs whose device memory is
 * reserved by another allocator (e.g. a framework's caching pool that holds the free
 * memory), or that must not pay the device-wide synchronisation cudaFree implies.
 *  - Workspace: one fixed 16 MiB array compiled into the library.  Every GPU that loads the
 *    library holds it until the process exits.  A call whose workspace (8 bytes per sample
 *    for each q and each (degree, window) candidate, twice, plus small tables) exceeds
 *    16 MiB returns LRT_EINVAL with the sizes in lrtddft_last_error.
 *  - The first call for a context on a device looks up the array's device address on that
 *    device (cudaGetSymbolAddress, with the device current); make that first call before
 *    any stream capture.
 *  - All calls share the array, which keeps the last call's contents; each call clears the
 *    part it uses before its kernels run.  Calls whose work overlaps on the GPU (several host
 *    threads, contexts or streams) race on the array: serialise them. */
lrt_status lrtddft_attenuate_noalloc(lrt_ctx* ctx, const lrt_atten_params* params, double* Sp,
                                     lrt_atten_report* report);

/* ---- The eta-convergence test from the Kubo-Greenwood conductivity (App. A.3).
 * Optical limit q -> 0 of the interband response on the k mesh and orbitals of q index 0
 * (trace/3 of the conductivity tensor), FP64:
 *   L(w) = (2/(N_k Omega)) sum_{k,n,n'} w_nk w_n'k (f_nk - f_n'k) (|p_nn'|^2/3) / Delta^2
 *          / (w + Delta + i eta),  p_nn' = <nk|-i grad|n'k>,  Delta = eps_nk - eps_n'k
 *   sigma_KG = i w L,  eps_KG = 1 + 4 pi i sigma_KG/w (Eq. 11),  chi*_KG = 1/eps_KG - 1
 *   (Eqs. 10, 12),  S*_KG = -Im chi*_KG / (pi n (1 - e^{-w/T})) (Eq. 13; at w = 0 its exact
 *   limit), and F*_KG (Eq. 14) by the fold of Eq. 1.
 * For eta [n_eta] (strictly increasing, Ha; 1..64): sigma [n_eta][nw] complex, S [n_eta][nw],
 * F [n_eta][ntau] at the caller's tau, metrics [n_eta][5] as itcf_laplace (each may be NULL),
 * and *eta_ref, the reference eta by the rule of lrtddft_eta_scan with tolerance tol.  Host
 * buffers.  Needs only the context's ground state. */
lrt_status lrtddft_kubo_greenwood(lrt_ctx* ctx, int n_eta, const double* eta, int ntau,
                                  const double* tau, double tol, double* sigma, double* S,
                                  double* F, double* metrics, int* eta_ref);
/* After lrtddft_kubo_greenwood: the attenuation (as lrtddft_attenuate) of S*_KG at the reference
 * eta, Sp [nw] and report [1], and, if out is not NULL, the filtered response at the samples
 * w >= 0 as lrtddft_dielectric returns it with v(q) chi = chi*: out [N][8] = chi*, 1/eps, eps,
 * sigma (each re, im).  LRT_ESTATE before a scan. */
lrt_status lrtddft_kubo_greenwood_attenuate(lrt_ctx* ctx, const lrt_atten_params* params, double* Sp,
                                            lrt_atten_report* report, double* out);

/* ---- instrumentation ---- */

/* Reset the counters below and turn the CUDA-event timing of the chi0 contraction and
 * pair-density kernel launches on (enable = 1) or off (0).  Events are recorded on the stream
 * each launch is enqueued on. */
lrt_status lrtddft_profile(lrt_ctx* ctx, int enable);
/* Synchronises the device and reads the counters since the last lrtddft_profile call:
 * out[0] kernels launched by the library, out[1] chi0 contraction launches timed,
 * out[2] their total device time in ms, out[3] pair-density launches timed, out[4] their
 * total ms, out[5] chi0 complex MACs of the timed contractions (N_G^2 N_w N_p summed, with
 * the caller's N_w), out[6..7] reserved (0). */
lrt_status lrtddft_profile_read(lrt_ctx* ctx, double out[8]);

/* Measured FP64 fused-multiply-add rate of a device's CUDA cores, TFLOP/s (2 flops per FMA):
 * a loop of independent FMAs on every SM, best of 5 launches timed with CUDA events.  The
 * roofline of the FP64 chi0 form, which runs on that pipe. */
lrt_status lrtddft_measure_fp64(int device, double* tflops);

/* ---- test and debug hooks ---- */

/* Replace the orbitals of q index iq: eps [2][nk][nb] ascending per k point (k mesh then k+q
 * mesh), coeff [2][nk][nb][npw] complex on the context's padded basis order (see
 * lrtddft_get_basis), occ [2][nk][nb] or NULL (Fermi-Dirac with a new mu).  The band weights
 * are recomputed from eps.
 * Host pointers. */
lrt_status lrtddft_set_orbitals(lrt_ctx* ctx, int iq, const double* eps, const double* coeff,
                                const double* occ);
/* The same replacement, pipelined: the coefficients are copied on a stream of the context's own
 * while earlier work runs, into a second set of orbital buffers (2 N_k N_b N_pw complex per q,
 * allocated on first use), and take effect at the next call that uses the orbitals of iq
 * (lrtddft_chi0_assemble over iq, whose stream then waits for the copy, or any call reading
 * the ground state of iq); results of the current orbitals (chi0, chi, S, F, derivatives) stay
 * valid until then.  eps and occ are read before the call returns.  coeff must stay unchanged
 * until that adopting call's stream has passed it (e.g. until a later call returning results
 * to the host has returned), and should be page-locked host memory for the copy to overlap
 * kernels (pageable memory is copied correctly, without overlap).  A later lrtddft_set_orbitals
 * of iq drops a pending upload.  Errors as lrtddft_set_orbitals.  Host pointers. */
lrt_status lrtddft_set_orbitals_async(lrt_ctx* ctx, int iq, const double* eps, const double* coeff,
                                      const double* occ);
/* Orbital coefficients of q index iq: coeff [2][nk][nb][npw] complex (the layout
 * lrtddft_set_orbitals takes). */
lrt_status lrtddft_get_orbitals(const lrt_ctx* ctx, int iq, double* coeff);
/* Miller indices of the padded basis of q index iq: miller [2][nk][npw][3] (int32; padding
 * rows hold INT32_MIN), npw_k [2][nk]. */
lrt_status lrtddft_get_basis(const lrt_ctx* ctx, int iq, int32_t* miller, int32_t* npw_k);
/* Eigenvalues [2][nk][nb], occupations [2][nk][nb], band weights [2][nk][nb] and mu of q
 * index iq (each pointer may be NULL); nb = lrtddft_query out[3] >= nbands.  The weights are
 * 1 for the lowest nbands bands and 0 above, except on a degenerate multiplet (eigenvalues
 * within 1e-6 Ha of band nbands-1) that the band cut splits: there each of its m members
 * carries j/m (j members below the cut), so that the kept band projector does not depend on
 * the eigensolver's choice of basis inside the multiplet.  A pair enters chi0 with
 * df_p = w_nk w_n'k+q (f_nk - f_n'k+q). */
lrt_status lrtddft_get_ground_state(const lrt_ctx* ctx, int iq, double* eps, double* occ,
                                    double* weights, double* mu);
/* Response G-set of q index iq: miller [nG][3] (G = 0 first) and K_GG [nG]. */
lrt_status lrtddft_get_gset(const lrt_ctx* ctx, int iq, int32_t* miller, double* K);
/* chi0 of q index iq: [nw_int][nG][nG] complex, at the internal frequencies
 * (lrtddft_get_frequencies).  Requires chi0_assemble on iq. */
lrt_status lrtddft_get_chi0(const lrt_ctx* ctx, int iq, double* chi0);
/* Pair densities rho_p(G) of q index iq as the contraction receives them: [N_p][nG] complex,
 * p = (k nb + n) nb + n', computed by the context's pair-density kernel (FP64 for the FP64
 * precision; FP32 on the tensor cores, or the FP32 SIMT kernel under LRT_TUNE_PAIR_SIMT, for
 * the split precisions).  Test hook; depends on the orbitals' phases (not gauge invariant). */
lrt_status lrtddft_get_pair_densities(lrt_ctx* ctx, int iq, double* rho);
/* chi_{G,0} of q index iq: [nw_int][nG] complex.  Requires dyson_solve on iq. */
lrt_status lrtddft_get_chi_col0(const lrt_ctx* ctx, int iq, double* chi);
/* Internal frequencies [nw_int] and the index of the w = 0 column. */
lrt_status lrtddft_get_frequencies(const lrt_ctx* ctx, double* freqs, int* hcol);
/* The row plan of the split-precision contraction for nG response G vectors (1..4096; host
 * only, no device work).  The Hermitian-split rows (Re and Im of rho(G) rho*(G') for G <= G')
 * are cut into sub-blocks of 16 row pairs, 8 per 256-row super-tile: a 4 x 4 block of G quads,
 * or a list of 16 pairs where a quad block would hold padding.  n_st: super-tiles (the least
 * any covering has, ceil(nG (nG + 1) / 256)); n_list: list sub-blocks; max_blocks: the most
 * 8-G blocks of pair densities one super-tile reads (at most 6); rp [nG][nG] (int32, or NULL):
 * the row pair (rows 2 rp, 2 rp + 1) of (min(G, G'), max(G, G')).  LRT_EINVAL on a NULL
 * output or nG out of range. */
lrt_status lrtddft_row_plan(int nG, int* n_st, int* n_list, int* max_blocks, int32_t* rp);

#ifdef __cplusplus
}
#endif
#endif /* LRTDDFT_H */
