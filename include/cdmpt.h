/*
 * cdmpt.h - C ABI of the GB300 (sm_103a) canonical density matrix
 * perturbation theory library (libcdmpt.so).
 *
 * The library evaluates, on one GPU, the hot path of canonical density
 * matrix perturbation theory (Niklasson, Rubensson, Rudberg, Cawkwell):
 *
 *   - the recursive Fermi-operator expansion, Eq. (Rec_F_2):
 *       X_0 = I/2 - 2^-(n+2) beta (H0 - mu I),
 *       X_k = X_{k-1}^2 [X_{k-1}^2 + (I - X_{k-1})^2]^-1,  k = 1..n,
 *     each step a linear solve T X_k = X_{k-1}^2 with
 *     T = 2 X_{k-1}(X_{k-1} - I) + I, by conjugate gradients warm-started
 *     from the previous iterate (Sec. II, Algorithm 1);
 *   - the first-order response X^(1) carried through every step with the
 *     same system matrix T (Algorithm 1, order 1);
 *   - the canonical constraint Tr P0 = N_occ on mu (Newton steps on the
 *     occupation, Eq. NewtRaphs) and Tr P1 = 0 on mu1 (Sec. II);
 *   - the polarizability alpha = -2 Tr[P1 H1] (the n+1 rule, Eq. Resp_0).
 *
 * Internally the recursion runs on the deviation Z = 2X - I, for which a
 * step is Z_{k+1} = 2 (I + Z_k^2)^-1 Z_k; P0 = (I + Z_n)/2, P1 = Z^(1)_n / 2.
 *
 * Conventions for every entry point:
 *   - Matrices are dense, row-major, symmetric, N x N with leading
 *     dimension N unless an ld argument says otherwise. Stacks of D
 *     matrices are contiguous, D * N * N.
 *   - Device pointers are CUDA global-memory addresses on the current
 *     device. Host pointers are ordinary CPU memory.
 *   - The caller owns every buffer it passes; the library copies what it
 *     keeps. The handle owns its device workspace and frees it in
 *     cdmpt_destroy.
 *   - Every call returns a cdmpt_status; no C++ exception crosses the ABI.
 *     On failure cdmpt_last_error() describes the cause.
 *   - A handle is not thread-safe: use it from one host thread and one
 *     CUDA stream at a time.
 */
#ifndef CDMPT_H
#define CDMPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CDMPT_VERSION_MAJOR 0
#define CDMPT_VERSION_MINOR 1

typedef enum {
    CDMPT_OK = 0,
    CDMPT_ERR_ARG = 1,            /* invalid argument (size, pointer, symmetry) */
    CDMPT_ERR_RANGE = 2,          /* beta * spectral width / 2^(n+1) >= 1: X_0 leaves [0,1] */
    CDMPT_ERR_NO_CONVERGENCE = 3, /* occupation (mu) loop did not converge */
    CDMPT_ERR_CG_MAXITER = 4,     /* a conjugate-gradient solve hit its iteration cap */
    CDMPT_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
    CDMPT_ERR_CUDA = 6,           /* a CUDA runtime call failed */
    CDMPT_ERR_OOM = 7,            /* device allocation failed */
    CDMPT_ERR_UNSUPPORTED = 8     /* feature not available on this device / build */
} cdmpt_status;

typedef enum {
    CDMPT_FP64 = 0,       /* FP64 storage, FP64 products (tensor-core Ozaki slicing into seven
                             BF16 digits on sm_103, or CUDA-core DFMA with CDMPT_GEMM_SIMT) */
    CDMPT_FP32 = 1,       /* FP32 storage, FP32-accurate products (3xTF32 on tcgen05 by default) */
    CDMPT_MIXED_TF32 = 2, /* one-pass TF32 products for the occupation sweeps; iterative
                             refinement of the pair-stored (hi + lo FP32) trajectory with
                             split-TF32 residuals on the early steps and FP64-class
                             (Ozaki-sliced BF16) residuals on the late ones (fp64_residual);
                             split-TF32 response right-hand sides */
    CDMPT_MIXED_BF16 = 3  /* as MIXED_TF32 with BF16 products (FP32 accumulation) for the
                             occupation sweeps */
} cdmpt_precision;

typedef enum {
    CDMPT_GEMM_AUTO = 0,      /* engine chosen from the precision */
    CDMPT_GEMM_SIMT = 1,      /* CUDA-core FFMA/DFMA tiles */
    CDMPT_GEMM_TC_TF32 = 2,   /* tcgen05 kind::tf32, one pass, FP32 accumulate in TMEM */
    CDMPT_GEMM_TC_3XTF32 = 3, /* tcgen05 kind::tf32, hi/lo split, three passes */
    CDMPT_GEMM_TC_BF16 = 4,   /* tcgen05 kind::f16 on operands rounded to BF16, one pass */
    CDMPT_GEMM_TC_OZAKI = 5   /* Ozaki-sliced BF16 digit products on tcgen05: the FP64-class
                                 refinement residuals of the mixed precisions (pair-stored
                                 operands, cdmpt_gemm_pair; statistics only there), and every
                                 product of the FP64 precision (seven digits, cdmpt_gemm_f64_tc;
                                 the default for FP64 on sm_103) */
} cdmpt_gemm_engine;

typedef struct {
    int precision;      /* cdmpt_precision */
    int gemm_engine;    /* cdmpt_gemm_engine. FP64 storage: AUTO or TC_OZAKI (FP64 Ozaki
                           products on the tensor cores) or SIMT (CUDA-core DFMA) */
    double cg_tol;      /* CG stop: ||R||_F <= cg_tol * ||RHS||_F; <= 0 selects the default */
    int cg_maxit;       /* CG iteration cap per solve */
    int refine_rounds;  /* residual-refinement rounds (MIXED_* only) */
    double occ_tol;     /* stop when |Tr P0 - N_occ| <= occ_tol; <= 0 selects N * 1e-12 (FP64)
                           or N * 1e-7 (otherwise) */
    int mu_maxit;       /* cap on occupation sweeps */
    int have_mu_guess;  /* 1: start Newton from mu_guess; 0: start from Tr(H0)/N */
    double mu_guess;
    int profile;        /* 1: time every GEMM launch with CUDA events (see cdmpt_stats) */
    void* stream;       /* cudaStream_t for all work of this handle; NULL = default stream */
    int grand_canonical; /* 1: grand-canonical solve at the fixed mu = mu_guess (needs
                            have_mu_guess): one occupation sweep, no mu update, mu1 = 0 (the
                            fixed-mu scheme Sec. II mentions beside Algorithm 1); nocc is
                            ignored. Batches are always canonical. */
    int ckpt_stride;    /* trajectory checkpoints (FP64 and FP32 precisions): 0 keeps every
                           Z_k; s > 0 keeps Z_k for k a multiple of s, Z_n and W_0, and
                           recomputes the other steps one segment of s steps at a time when
                           the response, the adjoint or a higher order needs them; -1 selects
                           s = ceil(sqrt(n)), which keeps about 3 sqrt(n) matrices instead of
                           2n. Mixed precisions return ERR_ARG for a nonzero value. */
    int fd_exact;       /* 1: start the recursion from Z_0 = tanh(-beta (H0 - mu I) / 2^(n+1))
                           (X_0 = (I + Z_0) / 2) instead of the linear X_0 of Eq. Rec_F_2. The
                           n steps then give P0 = [exp(beta (H0 - mu I)) + I]^-1 exactly (the
                           Fermi-Dirac function, Eq. Rec_F_1) rather than the n-step
                           approximation, and dP0/dmu = beta P0 (I - P0) holds exactly. tanh
                           is its odd Taylor series (converges since |Y| < 1 < pi/2), a few
                           products on the Gershgorin interval. Every derivative follows the
                           start: the response orders through the Taylor coefficients of tanh
                           along H(lambda), the adjoint through its (self-adjoint) tangent,
                           and cdmpt_free_energy gives the Fermi-Dirac Mermin free energy,
                           whose canonical gradient is P0. cdmpt_batch_create refuses it
                           (ERR_UNSUPPORTED). */
    double screen_tau;  /* > 0: block-sparse products (Sec. VI, Fig. 3: thresholded algebra
                           for linear scaling). Each product X Y^T of the solve and of its
                           derivatives drops the k-slice terms X_IK Y_JK^T of 128 x 32 tiles
                           whose Frobenius norms satisfy ||X_IK|| ||Y_JK|| <= screen_tau, so
                           the error of an output tile is at most screen_tau times the
                           number of dropped slices, and the work follows the number of
                           blocks above the threshold. Storage stays dense. FP32 and
                           MIXED_TF32 with the tcgen05 engines only (ERR_ARG otherwise);
                           0 (the default) keeps every product dense. */
    int fp64_residual;  /* MIXED_* only: the refinement that recovers accuracy keeps the
                           0th-order trajectory Z_0 .. Z_n as FP32 pairs (about 48 bits).
                           Once the split-TF32 passes have settled, every further pass (and
                           the Newton steps on mu between them) forms the step residuals
                           r_k = 2 Z_k - Z_{k+1} A_k (Algorithm 1's per-step system) and step
                           matrices A_k = I + Z_k^2 of the chosen steps with Ozaki-sliced
                           BF16 tensor-core products accurate to about 2^-39 of the row
                           maxima (cdmpt_gemm_pair) instead of split-TF32 ones; the right
                           side I - Z_n^2 of dP0/dmu is formed the same way. 0 (default):
                           on the steps whose spectral bound tanh(2^k atanh rho) exceeds
                           1/2, rho = beta max|lambda - mu| / 2^(n+1) over the Gershgorin
                           interval (for the earlier steps the split-TF32 residual is already
                           that accurate, its error carrying the factor ||Z_k||^2); 1: on
                           every step; -1: no such pass (split-TF32 residuals only). */
} cdmpt_opts;

typedef struct {
    int N, D, n;                   /* sizes of the last solve */
    int mu_iterations;             /* occupation sweeps (0th-order recursions) */
    int cg_iterations_sweeps;      /* CG iterations summed over all sweeps */
    int cg_iterations_last_sweep;  /* CG iterations of the final sweep */
    int cg_iterations_response;    /* CG iterations of the response pass */
    int cg_iterations_q;           /* CG iterations of the dP/dmu solve */
    int cg_iterations_refine;      /* CG iterations of the refinement */
    int gemm_launches;             /* GEMM kernel launches */
    int kernel_launches;           /* all kernel launches of this library */
    double gemm_flops;             /* algorithmic GEMM flops, sum of 2 M N K */
    double tensor_flops;           /* flops issued to the tensor pipe (split passes counted) */
    double gemm_ms;                /* summed GEMM device time (profile = 1 only) */
    int gemm_timed;                /* GEMM launches that were timed */
    double mu, trace_P0, trace_Q;  /* final mu, Tr P0, Tr dP0/dmu */
    double occupation_error;       /* |Tr P0 - N_occ| + sum_d |Tr P1_d| */
    double seconds;                /* host wall time of the last solve */
    double engine_ms[6];           /* GEMM device time per cdmpt_gemm_engine (profile = 1) */
    int engine_launches[6];        /* timed GEMM launches per engine */
    double engine_flops[6];        /* algorithmic flops of those launches */
    int cg_iterations_recompute;   /* CG iterations spent recomputing checkpointed segments */
    int checkpoint_stride;         /* stride in use (0: whole trajectory stored) */
    double screen_slices_computed; /* screened products of the last solve: 128 x 32 k-slices */
    double screen_slices_examined; /* multiplied, and all slices of their output tiles */
    int fp64_residual_passes;      /* refinement passes with Ozaki-sliced (FP64-class) residuals */
    int fp64_residual_first_step;  /* first step k they covered (n: none) */
    int refine_passes;             /* refinement passes of the mixed precisions, all kinds */
    double phase_ms[5];            /* device time of the solve's phases (profile = 1): occupation
                                      sweeps, refinement, first-order response, dP0/dmu with mu1
                                      and alpha, output of P0 and P1 */
} cdmpt_stats;

typedef struct cdmpt_handle cdmpt_handle;

/* Library version as (major << 16) | minor. */
int cdmpt_version(void);

/* Fill *opts with defaults: FP32 precision, automatic engine, cg_tol 1e-7
 * (FP32) / 1e-13 (FP64), cg_maxit 200, refine_rounds 2, mu_maxit 60,
 * profile 0, default stream. Returns CDMPT_ERR_ARG if opts is NULL. */
cdmpt_status cdmpt_default_opts(cdmpt_opts* opts);

/* Create a handle bound to the current CUDA device. opts may be NULL for
 * defaults; the struct is copied. *out receives the handle.
 * Errors: ERR_ARG (out NULL, bad precision/engine), ERR_UNSUPPORTED (a
 * tcgen05 engine on a device that is not sm_103), ERR_CUDA. */
cdmpt_status cdmpt_create(const cdmpt_opts* opts, cdmpt_handle** out);

/* Replace the options of an existing handle (stream, tolerances, precision). */
cdmpt_status cdmpt_set_opts(cdmpt_handle* h, const cdmpt_opts* opts);

/* Non-orthogonal basis (Sec. IV, Eq. Fermi_D): set the overlap matrix S (N x N,
 * symmetric positive definite, row-major FP64, host or device per on_device).
 * The handle computes the Loewdin factor Z = S^(-1/2) on the device by the
 * coupled Newton-Schulz iteration (products only, FP64, stopped when
 * ||Z Y - I||_F / sqrt(N) < 1e-12 plus one more step), so that Z^T S Z = I.
 * From then on cdmpt_set_H takes the non-orthogonal F (as H0) and h1 (as H1):
 * the solve works on F_perp = Z F Z and h1_perp = Z h1 Z, and every N x N
 * output is mapped back with the same congruence: P0 -> D = Z P_perp Z
 * (Tr[D S] = N_occ), P1 -> D1, P2 and P3 -> D2 and D3, and the gradients of
 * cdmpt_vjp_P0 (whose G0 is then dL/dD), cdmpt_response2 and cdmpt_free_energy
 * become derivatives with respect to F. alpha, mu and the mu^(k) are basis
 * independent. S = NULL returns to the orthogonal mode. Either call discards
 * the stored Hamiltonian, so cdmpt_set_H must follow. Batches are always
 * orthogonal. Errors: ERR_ARG (N < 1, no positive Gershgorin bound),
 * ERR_NO_CONVERGENCE (S not positive definite or too ill-conditioned for 200
 * iterations), ERR_OOM, ERR_CUDA. */
cdmpt_status cdmpt_set_overlap(cdmpt_handle* h, int N, const double* S, int on_device);

/* Newton-Schulz iterations and final residual ||Z Y - I||_F / sqrt(N) of the
 * last cdmpt_set_overlap (0 and 0.0 in the orthogonal mode). Either pointer may
 * be NULL. Errors: ERR_ARG (h NULL). */
cdmpt_status cdmpt_get_overlap_info(const cdmpt_handle* h, int* iterations, double* residual);

/* Load the unperturbed Hamiltonian H0 (N x N) and D >= 0 perturbations H1
 * (D x N x N), Eq. (H_prt) with H^(1) = H1, in an orthogonal basis (Sec. II).
 * on_device = 0: host pointers; 1: device pointers. Both are copied into
 * handle-owned FP64 device storage, so the caller may free them afterwards.
 * Spectral bounds of H0 (Gershgorin discs) are computed on the device here.
 * Errors: ERR_ARG (N < 1, D < 0, H0 NULL, H1 NULL with D > 0), ERR_OOM,
 * ERR_CUDA. */
cdmpt_status cdmpt_set_H(cdmpt_handle* h, int N, const double* H0, int D, const double* H1,
                         int on_device);

/* A self-consistent charge (SCC) tight-binding model: a synthetic two-electron part
 * G(D) for the self-consistent layer of Sec. IV. With Mulliken charge fluctuations
 * dq_i = 2 (D S)_ii - q0_i (restricted: two electrons per orbital) and the potential
 * V = gamma dq, G(D)_ij = (S_ij / 2)(V_i + V_j) (S = I in the orthogonal mode).
 * G is the derivative of E(D) = 2 Tr[h D] + 1/2 dq^T gamma dq with respect to 2 D,
 * so Omega_SCF = E(D) - 2 T_e S[D_perp] is the variational free energy of Eq.
 * FreeE_tot for this model. */
typedef struct {
    const double* gamma;  /* N x N symmetric kernel of the charge fluctuations (FP64) */
    const double* q0;     /* N reference populations, or NULL for zero */
    double tol;           /* stop each loop when max_i |dq_out - dq_in| < tol;
                             <= 0: 1e-10 (FP64) or 1e-6 (otherwise) */
    int maxit;            /* iteration cap of each loop; <= 0: 200 */
    int history;          /* Anderson mixing depth; <= 0: 6 */
    double mix;           /* mixing weight of the residual; <= 0: 0.3 */
} cdmpt_scc_model;

/* Self-consistent canonical solve and its coupled-perturbed response (Sec. IV,
 * Eqs. FirstOrderPRT, Fermi_D, Resp_Omega) for the model above, in the basis set by
 * cdmpt_set_overlap (orthogonal if none).
 * SCF: the charges dq are iterated to a fixed point, each step a canonical solve
 * of F = hcore + G(D) (Tr[D S] = nocc) with Anderson mixing.
 * CPSCF: per direction d, D1 = R(h1_d + G(D1)) with R the canonical first-order
 * response on the converged trajectory; G is linear in D, so this is a linear
 * fixed point in dq1, iterated the same way.
 * Outputs (any may be NULL): D0 (N x N), D1 (D x N x N) in the caller's basis, host or device per
 * on_device; mu (1 double), mu1, omega1, omega2 (D doubles each, host) with
 * Omega_SCF^(m) = (2/m) Tr[h1 D^(m-1)]: omega1 = 2 Tr[h1 D0], omega2 = Tr[h1 D1].
 * iters (2 ints, host): SCF iterations and CPSCF iterations summed over directions.
 * Inputs hcore, h1 (D x N x N), model->gamma and model->q0 are host or device per
 * on_device. The handle's stored Hamiltonian is the last F afterwards.
 * Errors: ERR_ARG, ERR_NO_CONVERGENCE, ERR_CG_MAXITER, ERR_OOM, ERR_CUDA, and those of
 * cdmpt_solve. */
cdmpt_status cdmpt_scc_solve(cdmpt_handle* h, const cdmpt_scc_model* model, int N,
                             const double* hcore, int D, const double* h1, double beta,
                             double nocc, int n, double* D0, double* D1, double* mu, double* mu1,
                             double* omega1, double* omega2, int* iters, int on_device);

/* cdmpt_scc_solve plus the second-order self-consistent response (the hyperpolarizability
 * of Sec. IV): per direction, D2 = (1/2) d^2 D / d lambda^2, the canonical order-2 response
 * to F^(1) = h1 + G(D1) and F^(2) = G(D2) on the converged trajectory (one joint order-1-2
 * sweep per step of a second charge fixed point, iterated like the first), its shift mu2,
 * and Omega_SCF^(3) = (2/3) Tr[h1 D2] (Eq. Resp_Omega). D2: D x N x N in the caller's basis,
 * host or device per on_device; mu2, omega3: host arrays of D doubles; any may be NULL
 * (all NULL: no second order). iters[1] then counts both coupled-perturbed loops. */
cdmpt_status cdmpt_scc_solve2(cdmpt_handle* h, const cdmpt_scc_model* model, int N,
                              const double* hcore, int D, const double* h1, double beta,
                              double nocc, int n, double* D0, double* D1, double* mu, double* mu1,
                              double* omega1, double* omega2, double* D2, double* mu2,
                              double* omega3, int* iters, int on_device);

/* Higher terms of the perturbation, H(lambda) = H0 + lambda H1 + lambda^2 H2 +
 * lambda^3 H3 per direction (Eq. H_prt; Algorithm 1 starts order i from
 * X_0^(i) = -2^-(M+2) beta (H^(i) - mu^(i) I)). H2 and H3 are D x N x N FP64 (D and N
 * of the last cdmpt_set_H), host or device per on_device, either may be NULL (zero).
 * They enter cdmpt_response2 (P2, mu2, Omega^(3) = 1/3 (Tr[H1 P2] + 2 Tr[H2 P1] +
 * 3 Tr[H3 P0])) and cdmpt_response3 (P3, mu3, Omega^(4) = 1/4 (Tr[H1 P3] +
 * 2 Tr[H2 P2] + 3 Tr[H3 P1])), Eq. Resp_0; the first order and the solve do not
 * depend on them. While either is set, cdmpt_response2 refuses the polarizability
 * gradient (it is d alpha / d H0 for H^(2) = H^(3) = 0). cdmpt_set_H and
 * cdmpt_set_overlap clear them; in the non-orthogonal mode they are mapped like h1.
 * Errors: ERR_ARG (no directions set), ERR_OOM, ERR_CUDA. */
cdmpt_status cdmpt_set_H_orders(cdmpt_handle* h, const double* H2, const double* H3,
                                int on_device);

/* Canonical solve, Algorithm 1 to first order.
 * beta > 0: inverse temperature; nocc in (0, N): occupation; n >= 1:
 * recursion steps (M in the paper).
 * Outputs (any may be NULL to skip): P0 (N x N), P1 (D x N x N) as FP64,
 * host or device memory according to out_on_device; mu (1 double, host) and
 * mu1 (D doubles, host). With D = 0 only P0 and mu are produced.
 * Errors: ERR_ARG, ERR_RANGE (beta (lambda_max - lambda_min) / 2^(n+1) >= 1
 * for the Gershgorin bounds), ERR_NO_CONVERGENCE (occupation not reached in
 * mu_maxit sweeps), ERR_CG_MAXITER, ERR_TIMEOUT, ERR_CUDA, ERR_OOM. */
cdmpt_status cdmpt_solve(cdmpt_handle* h, double beta, double nocc, int n, double* P0,
                         double* P1, double* mu, double* mu1, int out_on_device);

/* Polarizability alpha_d = -2 Tr[P1_d H1_d] of the last solve, for d < D,
 * written to alpha (D doubles, host). This is -4 Omega^(2) of Eq. (Resp_0)
 * with H^(2) = 0. Errors: ERR_ARG if no solve has completed. */
cdmpt_status cdmpt_polarizability(cdmpt_handle* h, double* alpha);

/* Adjoint (vector-Jacobian product) of the last cdmpt_solve on this handle:
 * gradH0 = d Tr[G0 P0] / d H0, the gradient of any scalar loss L(P0) with
 * dL/dP0 = G0, under the canonical constraint Tr P0 = N_occ (mu follows H0).
 * Computed by a reverse sweep through the stored recursion trajectory
 * (Eq. Rec_F_2 differentiated step by step, one linear solve with the same
 * step matrix T_k per step, Sec. II), then the chemical-potential term.
 * The Hessian of the free energy is symmetric, so gradH0 equals the canonical
 * first-order response P1 for the perturbation H1 = sym(G0) (App. B).
 * G0, gradH0: N x N FP64, host or device per on_device. Must follow a
 * successful cdmpt_solve on this handle (its trajectory is reused).
 * Errors: ERR_ARG (no solve yet, NULL pointers), ERR_CG_MAXITER, ERR_CUDA. */
cdmpt_status cdmpt_vjp_P0(cdmpt_handle* h, const double* G0, double* gradH0, int on_device);

/* First-order canonical response of the last solve to other perturbations: D
 * directions H1_d (D x N x N FP64, host or device per on_device), answered on the
 * stored trajectory without a new solve (every order and direction shares the step
 * matrices T_k, Sec. II). P1_d (D x N x N, may be NULL) with mu1_d from Tr P1_d = 0,
 * Omega^(2)_d = 1/2 Tr[H1_d P1_d] (Eq. Resp_0) and the polarizability
 * alpha_d = -2 Tr[H1_d P1_d] = -4 Omega^(2)_d, host arrays of D doubles (each may
 * be NULL). In the non-orthogonal mode H1 is h1 and P1 is D1.
 * Errors: ERR_ARG (no solve yet, D outside 1..16, H1 NULL), ERR_CG_MAXITER,
 * ERR_NO_CONVERGENCE, ERR_OOM, ERR_CUDA. */
cdmpt_status cdmpt_response1(cdmpt_handle* h, int D, const double* H1, double* P1, double* mu1,
                             double* omega2, double* alpha, int on_device);

/* Second-order canonical response of the last solve, per direction d of H1:
 * P2_d = (1/2) d^2 P / d lambda_d^2 of P(H0 + lambda_d H1_d) (Algorithm 1, the
 * order-2 line, with H^(2) = 0), with the second-order chemical-potential
 * shift mu2_d fixed by Tr P2_d = 0 (the canonical condition of Algorithm 1).
 * Also the gradient of L = sum_d w_d alpha_d, alpha_d = -2 Tr(P1_d H1_d), with
 * respect to H0: dL/dH0 = -4 sum_d w_d P2_d. This follows from the symmetry of
 * the third derivatives of the canonical free energy, whose H0-gradient is P0
 * (App. B), and holds exactly for the recursion's own occupation function.
 * Also Omega^(3)_d = (1/3) Tr[H1_d P2_d], the third-order free-energy term of
 * Eq. (Resp_0) with H^(1) = H1_d (the n+1 rule: P^(2) suffices for it).
 * w: host array of D weights, or NULL for all ones.
 * P2: D x N x N (row-major FP64), may be NULL. mu2, omega3: host arrays of D
 * doubles, may be NULL. gradH0: N x N, may be NULL. P2 and gradH0 are host or device
 * memory per on_device. The call runs, per direction, one joint forward sweep
 * of orders 1 and 2 with the known mu1 (eight products and two CG solves per
 * step) in the precision of the solve.
 * Errors: ERR_ARG (no solve yet, no directions), ERR_CG_MAXITER,
 * ERR_NO_CONVERGENCE, ERR_OOM, ERR_CUDA. */
cdmpt_status cdmpt_response2(cdmpt_handle* h, const double* w, double* P2, double* mu2,
                             double* omega3, double* gradH0, int on_device);

/* Third-order canonical response of the last solve, per direction d of H1:
 * P3_d = (1/6) d^3 P / d lambda_d^3 of P(H0 + lambda_d H1_d) (Algorithm 1, the
 * order-3 line, with H^(2) = H^(3) = 0). mu2_d comes from an order-2 pass and
 * mu3_d from Tr P3_d = 0 (the canonical conditions of Algorithm 1). Also
 * Omega^(4)_d = (1/4) Tr[H1_d P3_d], the fourth-order free-energy term of
 * Eq. (Resp_0) (the n+1 rule: P^(3) suffices for it).
 * P3: D x N x N (row-major FP64), host or device memory per on_device, may be
 * NULL. mu3, omega4: host arrays of D doubles, may be NULL. The call runs, per
 * direction, one joint sweep of orders 1-2 and one of orders 1-3 (every order
 * solved with the step matrix of the 0th order) in the precision of the solve.
 * Errors: ERR_ARG (no solve yet, no directions), ERR_CG_MAXITER,
 * ERR_NO_CONVERGENCE, ERR_OOM, ERR_CUDA. */
cdmpt_status cdmpt_response3(cdmpt_handle* h, double* P3, double* mu3, double* omega4,
                             int on_device);

/* Free energy of the last solve, Omega = Tr[P0 H0] - T_e S[P0] with the
 * entropy S[P] = -Tr[P ln P + (I - P) ln(I - P)] (Eqs. FreeE, SED; k_B = 1,
 * T_e = 1/beta), for the recursion's own P0 (the n-step function of Eq.
 * Rec_F_2), and optionally its gradient gradH0 = dOmega/dH0 under the solve's
 * constraint (canonical: Tr P0 = N_occ held, mu follows H0; grand canonical:
 * mu held). No eigenvalues are used: per level 1 - x_{k+1} = (1 - x_k)^2 /
 * (x_k^2 + (1 - x_k)^2), so ln det(I - P0) is a weighted sum of the
 * log-determinants of I - Z_0 and of the step matrices A_k = I + Z_k^2, each
 * found by one CG solve and a short series; the entropy's remaining term
 * needs atanh(Z_0) - Z_0, a series in Z_0^2. For the Fermi-Dirac function the
 * canonical gradient would be P0 (App. B); for the n-step function it is P0
 * plus one adjoint sweep (as cdmpt_vjp_P0) of mu I + T_e ln(P0 (I - P0)^-1) -
 * (H0 - mu I), a correction of the size of the recursion's truncation error.
 * omega: host double, may be NULL. gradH0: N x N FP64, host or device per
 * on_device, may be NULL (then no adjoint sweep runs). Must follow a
 * successful cdmpt_solve on this handle.
 * Errors: ERR_ARG (no solve yet), ERR_CG_MAXITER, ERR_OOM, ERR_CUDA. */
cdmpt_status cdmpt_free_energy(cdmpt_handle* h, double* omega, double* gradH0, int on_device);

/* Spectral interval of a symmetric matrix from Gershgorin discs:
 * bounds[0] = min_i (H_ii - sum_{j != i} |H_ij|), bounds[1] = max_i (H_ii + sum_{j != i} |H_ij|).
 * Every eigenvalue of H lies in [bounds[0], bounds[1]]. cdmpt_solve needs
 * beta (bounds[1] - bounds[0]) / 2^(n+1) < 1 so that X_0 of Eq. (Rec_F_2) keeps
 * its spectrum inside [0, 1]; this call lets a caller pick n before solving.
 * H: N x N FP64 device array with leading dimension ldh >= N. bounds: 2
 * doubles of device memory. Uses 16 N bytes of temporary device memory
 * (stream-ordered allocation). Asynchronous on stream.
 * Errors: ERR_ARG (N < 1, ldh < N, NULL pointers), ERR_CUDA. */
cdmpt_status cdmpt_spectral_bounds(const double* H, int N, int ldh, double* bounds, void* stream);

/* Allocation-free cdmpt_spectral_bounds, for callers that must not allocate
 * device memory: code that runs while a stream is being captured into a CUDA
 * graph (plain cudaMalloc is not allowed there), code that runs under an
 * allocator which already owns the whole device memory budget, and latency-
 * critical loops where cudaFree would synchronize the device. The paper has
 * no counterpart; this is an interface convenience.
 * Same arguments, results and asynchrony as cdmpt_spectral_bounds; the caller
 * still passes H and bounds. The per-row scratch sits in a fixed 512 KiB
 * array of the library's static device memory, so N may be at most 32768
 * (larger N returns ERR_ARG). That array is held on every GPU that loads the
 * library until the process exits, and every call shares it: calls whose
 * kernels overlap on the GPU (different streams, or different host threads)
 * race on it and must be serialised by the caller. The first call on a
 * device looks up the array's device address; make that first call before
 * any stream capture begins. The address is kept for the life of the process:
 * after cudaDeviceReset (or any reset of the device's primary context) the
 * library's module is reloaded elsewhere and this entry point must not be
 * called again on that device. No call allocates or frees memory.
 * Errors: ERR_ARG (N < 1, N > 32768, ldh < N, NULL pointers), ERR_CUDA. */
cdmpt_status cdmpt_spectral_bounds_noalloc(const double* H, int N, int ldh, double* bounds,
                                           void* stream);

/* Statistics of the last solve (copied into *st). */
cdmpt_status cdmpt_get_stats(const cdmpt_handle* h, cdmpt_stats* st);

/* Human-readable description of the last error of this handle ("" if none). */
const char* cdmpt_last_error(const cdmpt_handle* h);

/* Free the handle and all device memory it owns. NULL is ignored. */
void cdmpt_destroy(cdmpt_handle* h);

/* ---------------------------------------------------------------- batches
 * Many independent canonical solves of uneven size N_b (b < B), each with the
 * same number D of perturbation directions, advanced in lockstep: every
 * product of a recursion step is one grouped persistent tcgen05 launch over
 * all systems, every vector update one grouped launch; each system keeps its
 * own CG scalars and chemical potential, and converged systems are skipped.
 * Storage FP32. CDMPT_FP32: split-TF32 products throughout. CDMPT_MIXED_TF32:
 * one-pass TF32 occupation sweeps, then refinement of every pair-stored
 * trajectory (split-TF32 passes, then FP64-class residuals on the late steps)
 * and a split-TF32 response, as in cdmpt_solve. In the refinement each system
 * switches to the FP64-class passes by itself, once its occupation error after
 * a split pass is within 1e-4 sqrt(N_b) (environment CDMPT_BATCH_HP_SWITCH; 0
 * switches after the first split pass), and finishes only in such a pass; the
 * FP64-class products of different systems run on CDMPT_BATCH_HP_LANES side
 * streams (default 8, at most 8).
 */
typedef struct cdmpt_batch cdmpt_batch;

/* Create a batch of B systems of sizes N[0..B-1] with D directions each.
 * Errors: ERR_ARG, ERR_UNSUPPORTED (precision other than FP32 or MIXED_TF32,
 * fd_exact, grand_canonical or screen_tau set, or no sm_103 device), ERR_OOM. */
cdmpt_status cdmpt_batch_create(const cdmpt_opts* opts, int B, const int* N, int D,
                                cdmpt_batch** out);

/* Load H0[b] (N_b x N_b) and H1[b] (D x N_b x N_b), FP64 row-major, host or
 * device pointers per on_device, and allocate the trajectory for n steps. */
cdmpt_status cdmpt_batch_set_H(cdmpt_batch* b, const double* const* H0, const double* const* H1,
                               int n, int on_device);

/* Solve all systems (Algorithm 1 to first order): beta[b], nocc[b] per
 * system; outputs per system (arrays of B pointers, entries may be NULL):
 * P0[b] (N_b x N_b), P1[b] (D x N_b x N_b); mu[B], mu1[B*D], alpha[B*D] on the
 * host (alpha_d = -2 Tr[P1_d H1_d]). Errors as for cdmpt_solve. */
cdmpt_status cdmpt_batch_solve(cdmpt_batch* b, const double* beta, const double* nocc, int n,
                               double* const* P0, double* const* P1, double* mu, double* mu1,
                               double* alpha, int out_on_device);

/* Statistics of the last batch solve (N holds B). */
cdmpt_status cdmpt_batch_get_stats(const cdmpt_batch* b, cdmpt_stats* st);

/* Tile autotuner and graph report of a batch. tile_n: the grouped kernel's
 * tile width chosen by timing each candidate on the batch's first product over
 * all systems; 0 before the first solve. The candidates are 128 x 128 and
 * 128 x 64 tiles on one SM, and 256 x 256 tiles on a cluster of two SMs for
 * the split-TF32 products (one-pass TF32 products then take 128 x 128 tiles);
 * all three accumulate the same k-chunks, so results agree to FP32 rounding. ms: an array of 3 that receives the measured time per launch
 * of the 128-, 64- and 256-column candidates (0 if not timed). graphs: 1 when
 * the CG iterations replay a captured CUDA graph (CDMPT_BATCH_GRAPH=0 turns
 * capture off; CDMPT_BATCH_TILE=64|128|256 fixes the tile width). Any pointer
 * may be NULL. Errors: ERR_ARG (b NULL). */
cdmpt_status cdmpt_batch_get_tuning(const cdmpt_batch* b, int* tile_n, double* ms, int* graphs);

/* Last error of the batch ("" if none). */
const char* cdmpt_batch_last_error(const cdmpt_batch* b);

/* Free the batch and its device memory. NULL is ignored. */
void cdmpt_batch_destroy(cdmpt_batch* b);

/*
 * Dense building block exposed for testing and benchmarking: the product of
 * one recursion step (Algorithm 1 forms every product X Y with Y symmetric).
 *
 *   D[m][n] = alpha * sum_k X[m][k] Y[n][k] + beta * C[m][n] + gamma * [m % diag_block == n]
 *
 * i.e. D = alpha X Y^T + beta C + gamma I_blocks, X: M x K, Y: Ncols x K, all
 * row-major device arrays (leading dimensions in elements; for the tcgen05
 * engines ldx and ldy must be multiples of 4 and X, Y 16-byte aligned).
 * trans_block > 0 writes (and reads C at) the transposed position inside
 * consecutive row blocks of height trans_block (requires Ncols == trans_block).
 * trans_block = -1 declares the result symmetric (M == Ncols; C and E
 * symmetric): the tensor-core engines then compute only the upper-triangular
 * tiles and mirror each off-diagonal tile, half the work; the CUDA-core
 * engines compute every element. Every 0th-order product of the recursion is
 * symmetric (functions of Z_k that commute).
 * dot != NULL accumulates sum_{m,n} D[m][n] * E[m][n] into *dot (device
 * double; E NULL means E = D). C may alias D. Asynchronous on stream.
 * engine: cdmpt_gemm_engine (AUTO = 3xTF32).
 * Errors: ERR_ARG, ERR_UNSUPPORTED, ERR_CUDA. */
cdmpt_status cdmpt_gemm_f32(int engine, int M, int Ncols, int K, const float* X, int ldx,
                            const float* Y, int ldy, float* D, int ldd, double alpha,
                            double beta, const float* C, int ldc, double gamma, int diag_block,
                            int trans_block, double* dot, const float* E, int lde, void* stream);

/* TF32 split of count FP32 values for the tensor-core engines:
 * hi = round_to_nearest_tf32(x), lo = round_to_nearest_tf32(x - hi), so that
 * hi + lo carries x to about 2^-22 relative (split-TF32 products).
 * count must be a multiple of 4; X, hi, lo 16-byte aligned device arrays. */
cdmpt_status cdmpt_split_tf32(const float* X, size_t count, float* hi, float* lo, void* stream);

/* cdmpt_gemm_f32 for operands already split by cdmpt_split_tf32 (Xhi/Xlo and
 * Yhi/Ylo share the leading dimensions ldx / ldy). engine TC_TF32 reads only
 * the hi arrays; TC_3XTF32 (or AUTO) all four. Lets a caller split an operand
 * once and reuse it over many products. */
cdmpt_status cdmpt_gemm_f32_split(int engine, int M, int Ncols, int K, const float* Xhi,
                                  const float* Xlo, int ldx, const float* Yhi, const float* Ylo,
                                  int ldy, float* D, int ldd, double alpha, double beta,
                                  const float* C, int ldc, double gamma, int diag_block,
                                  int trans_block, double* dot, const float* E, int lde,
                                  void* stream);

/* Product of pair-stored FP32 matrices (value = hi + lo) to about 31 bits, the building block
 * of the FP64-class refinement residual of the mixed precision (the per-step system of
 * Algorithm 1, T X = RHS, whose residual must be formed beyond FP32 accuracy). The paper has
 * no such kernel; the method is the error-free slicing of Ozaki et al. on tensor cores
 * (Mukunoki, Ozaki, Ogita and Imamura): each row of X and of Y is scaled by its own power of
 * two and cut into five signed 8-bit integer digits stored in BF16 (39 bits), the fifteen
 * digit products of weight above 2^-40 run on tcgen05 (kind::f16, FP32 accumulation in TMEM)
 * with the three leading groups summed exactly over every chunk of 256 k, and the epilogue
 * combines the exact sums in double-float:
 *   D + Dl = alpha (Xh + Xl)(Yh + Yl)^T + b1 (C1h + C1l) + b2 (C2h + C2l).
 * X is M x K, Y is Ncols x K (row-major device arrays, leading dimensions ldx, ldy multiples
 * of 8 elements, 16-byte aligned), C1/C2/D/Dl share ldc and ldd. Xl, Yl, C1h, C1l, C2h, C2l
 * and Dl may be NULL (a NULL low part is zero; a NULL C term is skipped; Dl NULL: D only).
 * alpha, b1 and b2 must be powers of two or zero, so every scaling is exact. The error of
 * D + Dl is about 2^-39 of max_k |x_ik| max_k |y_jk| times sqrt(K). K <= 32768. sym != 0
 * with Y the same arrays as X (Yh == Xh, Yl == Xl, Ncols == M) and symmetric C terms: only
 * the output tiles that meet the upper triangle are computed and every element with n >= m
 * is written at (m, n) and (n, m) (the products W = X X^T and I - X X^T of the mixed
 * refinement); otherwise sym is ignored. The digits of both operands (10 (M + Ncols) ld
 * bytes plus one int per row; once when Y is X) are allocated and freed stream-ordered on
 * the stream. Errors: ERR_ARG, ERR_UNSUPPORTED (not an sm_103 device), ERR_OOM, ERR_CUDA. */
cdmpt_status cdmpt_gemm_pair(int M, int Ncols, int K, const float* Xh, const float* Xl, int ldx,
                             const float* Yh, const float* Yl, int ldy, float* D, float* Dl,
                             int ldd, double alpha, double b1, const float* C1h, const float* C1l,
                             double b2, const float* C2h, const float* C2l, int ldc, int sym,
                             void* stream);

/* Check of the failure detection of the device waits (Sec. II of the paper names loss of
 * convergence as its only failure; the bounded waits of this library have no counterpart in
 * it). Every mbarrier wait of the tcgen05 kernels gives up after a time limit, records a code
 * in a device error word, and the next status check of the library returns
 * CDMPT_ERR_TIMEOUT. This call launches one CTA that waits, through that same bounded wait
 * with a limit of limit_ms milliseconds, on a barrier that nothing arrives on; no copy or
 * tensor-core operation is in flight. It returns CDMPT_ERR_TIMEOUT when the wait gave up as
 * designed (the error word is then cleared, so later calls are unaffected), CDMPT_OK never in
 * a working build, ERR_ARG for limit_ms outside (0, 1000], ERR_CUDA on a launch failure.
 * stream: cudaStream_t or NULL. */
cdmpt_status cdmpt_check_bounded_wait(double limit_ms, void* stream);

/* FP64 counterpart of cdmpt_gemm_f32 on CUDA cores (no alignment rule). */
cdmpt_status cdmpt_gemm_f64(int M, int Ncols, int K, const double* X, int ldx, const double* Y,
                            int ldy, double* D, int ldd, double alpha, double beta,
                            const double* C, int ldc, double gamma, int diag_block,
                            int trans_block, double* dot, const double* E, int lde,
                            void* stream);

/* The same product, arguments and semantics as cdmpt_gemm_f64 (trans_block = -1 is accepted
 * and computes every element), on the tensor cores by the error-free slicing of Ozaki et al.
 * (integer-accumulation form of Mukunoki, Ozaki, Ogita, Imamura, ISC 2020): each row of X and
 * Y is scaled by a power of two and cut into seven signed 8-bit digits (55 bits of the row's
 * largest element), the 28 digit products with weight at least 2^-48 run as BF16 tcgen05 MMAs
 * with FP32 accumulation, exact (integer) for the four leading weight groups, and the sums are
 * combined in FP64. Error: within about 2^-47 of |X_i| |Y_j| row maxima times K, against FP64
 * rounding of the exact product (tests: relative error below 1e-13 on random inputs). The
 * CUDA-core FP64 rate of this part is about 1.2 TFLOP/s; this path runs the FP64 precision's
 * products. Needs sm_103, K <= 16384; digits go to stream-ordered scratch of
 * 14 (M + Ncols) roundup(K, 8) bytes. Errors: ERR_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA. */
cdmpt_status cdmpt_gemm_f64_tc(int M, int Ncols, int K, const double* X, int ldx,
                               const double* Y, int ldy, double* D, int ldd, double alpha,
                               double beta, const double* C, int ldc, double gamma,
                               int diag_block, int trans_block, double* dot, const double* E,
                               int lde, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CDMPT_H */
