/*
 * afqmc.h -- C ABI of the B300 (sm_103a) phaseless-AFQMC hot path.
 *
 * The library propagates a batch of single-determinant walkers under a
 * Cholesky-factorised ab initio Hamiltonian with a single-determinant RHF/UHF
 * trial, and measures the mixed local energy.  Equation numbers refer to
 * arXiv:2406.16238 ("Improved Modularity and New Features in ipie"),
 * Section "Theory of AFQMC":
 *
 *   Eq. 2-3   H = sum h_pq a+_p a_q + 1/2 sum g_psqr a+_p a+_q a_r a_s,
 *             g_psqr = sum_gamma L^gamma_ps L^gamma_qr         (inputs h1e, chol)
 *   Eq. 4-6   H = v0 - 1/2 sum v_gamma^2, v_gamma = i sum L^gamma a+a
 *   Eq. 7-8   symmetric Trotter split and B(x) = e^{-dt/2 v0} e^{-sqrt(dt) x.v} e^{-dt/2 v0}
 *   Eq. 9     mixed energy estimator E = sum w E_loc                (afqmc_local_energy)
 *   Eq. 10-11 walker and weight update with shifted fields     (afqmc_propagate)
 *   Eq. 12    force bias with the mean-field shift
 *   Eq. 13-16 phaseless / hybrid importance function, overlap ratio, phase
 * plus the stabilisation and population control the driver performs each
 * block (Section "AFQMC driver"; afqmc_reortho, afqmc_popcontrol).
 *
 * Conventions (all calls):
 *   - Host arrays are row-major, float64, C-contiguous, owned by the caller
 *     and only read during the call (or written, for outputs).
 *   - Complex host arrays are interleaved (re, im) float64 pairs.
 *   - Device memory is never allocated by the library: the caller passes one
 *     device workspace of afqmc_workspace_size() bytes to afqmc_create and
 *     keeps it alive until afqmc_destroy.
 *   - Every call is ordered on the stream given in afqmc_params (NULL = the
 *     legacy default stream).  Calls that return host data synchronise that
 *     stream; afqmc_propagate, afqmc_reortho and afqmc_popcontrol only enqueue.
 *   - Errors are returned as afqmc_status; afqmc_last_error() gives a
 *     thread-local message.  Device-side conditions (a singular overlap, a
 *     non-finite weight, all weights zero) are recorded in a device status word
 *     and reported by the next synchronising call; the offending walkers get
 *     weight 0.  No call traps or aborts.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef AFQMC_H
#define AFQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afqmc_ctx afqmc_ctx;

typedef enum {
  AFQMC_OK = 0,
  AFQMC_EINVAL = 1,       /* bad argument (sizes, NaN input, non-symmetric L, ...) */
  AFQMC_ENOMEM = 2,       /* workspace smaller than afqmc_workspace_size() */
  AFQMC_ECUDA = 3,        /* a CUDA runtime call or launch failed */
  AFQMC_ESINGULAR = 4,    /* a walker's overlap matrix had a zero pivot (walker weight set to 0) */
  AFQMC_ENONFINITE = 5,   /* a walker's weight became NaN/Inf (walker weight set to 0) */
  AFQMC_ENOWALKERS = 6,   /* every walker weight is zero: population control cannot proceed */
  AFQMC_ETIMEOUT = 7      /* afqmc_synchronize gave up waiting */
} afqmc_status;

/* Arithmetic of the three large contractions (force bias, VHS build, exchange).
 * FP64: walkers complex128, every product and sum in binary64.
 * FP32: walkers complex64, contractions in binary32 (CUDA cores).
 * BF16: walkers complex64, contractions on the tcgen05 tensor cores with bf16
 *       operands and fp32 accumulation.  L is rounded to bf16 unscaled: bf16
 *       has the exponent range of fp32, so a per-gamma scale would change no
 *       rounding except in the subnormal range.
 * BF16X3: as BF16, but each fp32 operand is split into bf16 hi + lo parts and
 *       the products hi*hi + hi*lo + lo*hi are accumulated in fp32.
 * In every form the n x n overlap inverses and log-determinants, the phases
 * and weights, QR reorthogonalisation and the energy reductions are binary64. */
typedef enum { AFQMC_PREC_FP64 = 0, AFQMC_PREC_FP32 = 1, AFQMC_PREC_BF16 = 2, AFQMC_PREC_BF16X3 = 3 } afqmc_prec;

typedef struct {
  double dt;              /* imaginary time step Delta tau (> 0) */
  int32_t nwalkers;       /* walkers W (>= 1) */
  int32_t taylor_order;   /* terms of the exp(VHS) Taylor series (1..12; 6 usual) */
  double fb_cap;          /* |xbar_gamma| cap (<= 0: no cap) */
  uint64_t seed;          /* Philox4x32-10 key */
  int32_t prec;           /* afqmc_prec */
  int32_t reserved;       /* must be 0 */
  double e_trial;         /* energy shift E_T of the weights; NaN -> the trial's variational energy */
  void* stream;           /* cudaStream_t the context works on (NULL: default stream) */
} afqmc_params;

typedef struct {
  int32_t norb, naux, nalpha, nbeta, nwalkers;
  int32_t restricted;     /* 1: RHF trial with nalpha == nbeta, one spin block stored and propagated */
  int32_t prec;
  int32_t reserved;
  uint64_t step;          /* completed propagation steps (the Philox step counter) */
  double e_var;           /* <Psi_T|H|Psi_T> as measured by the library at create */
  double e_trial;         /* energy shift in use */
  double e_core_mf;       /* E_c = E0 - 1/2 sum lbar^2 (mean-field constant) */
  size_t workspace_bytes;
} afqmc_info;

/* Bytes of device workspace that afqmc_create needs for these sizes.
 * psiT [norb, nalpha+nbeta] (host) decides whether the trial is restricted. */
afqmc_status afqmc_workspace_size(int32_t norb, int32_t naux, int32_t nalpha, int32_t nbeta,
                                  const double* psiT, const afqmc_params* params, size_t* bytes);

/* Build a context (the paper's HamGeneric(h1e, chol, ecore) + SingleDet(psiT) +
 * AFQMC.build, Sections "Hamiltonian", "Trial wavefunctions", "AFQMC driver").
 *   h1e   [norb, norb]          one-body integrals h_pq, symmetric
 *   chol  [naux, norb, norb]    Cholesky vectors L^gamma_pq, each symmetric (Eq. 3)
 *   ecore                       constant E0
 *   psiT  [norb, nalpha+nbeta]  trial orbitals, alpha columns first (real)
 * Precomputes on the device: the mean-field shift lbar_gamma = Tr L^gamma P_T,
 * h_eff = h - 1/2 sum L L + sum lbar L and exp(-dt/2 h_eff), the half-rotated
 * Ltilde^gamma = Phi^T L^gamma and htilde = Phi^T h, and initialises every walker
 * to psiT with weight 1.  Limits: 1 <= nalpha, 0 <= nbeta, nalpha, nbeta <= min(norb, 64).
 * workspace: device pointer, 256-byte aligned, >= afqmc_workspace_size() bytes. */
afqmc_status afqmc_create(const double* h1e, const double* chol, double ecore,
                          int32_t norb, int32_t naux, int32_t nalpha, int32_t nbeta,
                          const double* psiT, const afqmc_params* params,
                          void* workspace, size_t workspace_bytes, afqmc_ctx** out);

/* Chunked construction, for Hamiltonians whose Cholesky tensor is too large to pass (or to hold in
 * binary64) at once.  afqmc_create_begin takes everything afqmc_create takes except chol, and
 * returns a context in set-up.  afqmc_add_cholesky then passes the vectors L^gamma for gamma =
 * gamma0 .. gamma0 + ngamma - 1 ([ngamma][norb][norb], each symmetric), in order and each exactly
 * once, as binary64 (dtype AFQMC_DTYPE_F64) or binary32 (AFQMC_DTYPE_F32) from host memory
 * (location AFQMC_HOST: copied through the workspace and checked on the host before the copy) or
 * from device memory (AFQMC_DEVICE: read in place, checked on the device; the check is reported by
 * afqmc_create_end).  The caller may reuse or free a chunk's memory when the call returns.
 * afqmc_create_end finishes the set-up once every vector has been passed: the mean-field shift
 * lbar_gamma = Tr L^gamma P_T, h_eff = h - 1/2 sum L L + sum lbar L, exp(-dt/2 h_eff) (all
 * accumulated on the device one chunk at a time, binary64 sums), the half-rotated tensors, the
 * walkers and E_var.  Until then every other call but afqmc_destroy rejects the context.  On an
 * error the context stays allocated; afqmc_destroy frees it.  afqmc_create is begin + one
 * afqmc_add_cholesky of every vector from host memory + end.  Set-up products that would cost more
 * than ~4e11 binary64 operations (sum L L, Ltilde) run in binary32 in the reduced-precision forms;
 * their sums over chunks stay binary64. */
#define AFQMC_DTYPE_F64 0
#define AFQMC_DTYPE_F32 1
#define AFQMC_DTYPE_C128 2   /* complex, interleaved (re, im) binary64: complex contexts only */
#define AFQMC_DTYPE_C64 3    /* complex, interleaved (re, im) binary32: complex contexts only */
#define AFQMC_HOST 0
#define AFQMC_DEVICE 1
afqmc_status afqmc_create_begin(const double* h1e, double ecore, int32_t norb, int32_t naux, int32_t nalpha,
                                int32_t nbeta, const double* psiT, const afqmc_params* params, void* workspace,
                                size_t workspace_bytes, afqmc_ctx** out);
afqmc_status afqmc_add_cholesky(afqmc_ctx* ctx, int32_t gamma0, int32_t ngamma, const void* chol, int32_t dtype,
                                int32_t location);
afqmc_status afqmc_create_end(afqmc_ctx* ctx);

/* Complex Hamiltonians (Section "Support of complex Cholesky vectors": complex orbitals, as with
 * Bloch orbitals, a magnetic field or spin-orbit coupling).  As afqmc_create_begin, with
 *   h1e   [norb][norb][2]          complex Hermitian one-body integrals (interleaved re, im)
 *   psiT  [norb][nalpha+nbeta][2]  complex trial orbitals
 *   naux                           the number of complex Cholesky vectors L^gamma, passed to
 *                                  afqmc_add_cholesky as AFQMC_DTYPE_C128 / C64 chunks
 *                                  [ngamma][norb][norb][2] with g_psqr = sum L_ps conj(L_rq)
 *                                  (the integrals' exchange symmetry (ps|qr) = (qr|ps) assumed).
 * Each vector gives two auxiliary fields with the Hermitian matrices A = (L + L^+) / 2 and
 * B = i (L - L^+) / 2, so the context draws 2 naux fields per walker (afqmc_get_fields, info.naux
 * report 2 naux); every formula of the real case holds with the trial's conjugate transpose.
 * Every precision form runs complex contexts.  The BF16 / BF16X3 forms realify each contraction along
 * K (a complex product as one real GEMM over [Re | Im] halves: the exchange, the VHS build over the
 * 2 naux fields and the propagation with complex E_h all take twice the K of a real context of the
 * same size).  The control variate takes real Hamiltonians only. */
afqmc_status afqmc_workspace_size_complex(int32_t norb, int32_t naux, int32_t nalpha, int32_t nbeta,
                                          const double* psiT, const afqmc_params* params, size_t* bytes);
afqmc_status afqmc_create_begin_complex(const double* h1e, double ecore, int32_t norb, int32_t naux, int32_t nalpha,
                                        int32_t nbeta, const double* psiT, const afqmc_params* params,
                                        void* workspace, size_t workspace_bytes, afqmc_ctx** out);

/* nsteps phaseless steps (Eqs. 10-16), each: Green's function / Theta and the
 * force bias at the current walkers (reused from afqmc_local_energy when it
 * was measured at the same walkers), Philox fields x with counter = the step,
 * shifted fields, VHS = -i sqrt(dt) sum_g (x - xbar)_g L^g, walkers
 * exp(-dt/2 h_eff) exp_Taylor(VHS) exp(-dt/2 h_eff) psi, new overlaps, weights
 * w |I| max(0, cos theta) exp(dt (E_T - E_c)).  Walkers of weight 0 are frozen. */
afqmc_status afqmc_propagate(afqmc_ctx* ctx, int32_t nsteps);

/* Mixed local energy (Eq. 9) of every walker and the estimator sums
 *   sums[4] = {ENumer = sum w Re E_L, EDenom = sum w, E1Body = sum w Re(E0 + E1),
 *              E2Body = sum w Re(J - K)}   (host, may be NULL)
 *   eloc    [nwalkers][3][2] (host, may be NULL): (E_L, E0 + E1, J - K) per walker.
 * Synchronises the stream when either output is non-NULL. */
afqmc_status afqmc_local_energy(afqmc_ctx* ctx, double* sums, double* eloc);

/* As afqmc_local_energy for the four sums only, without synchronising: the copy of sums[4] to
 * `sums_host` is enqueued on the context's stream after the energy kernels (use page-locked host
 * memory for an asynchronous copy).  The values are there once the stream has reached that point
 * (afqmc_synchronize or any stream synchronisation); device-side conditions are reported by the
 * next synchronising call. */
afqmc_status afqmc_local_energy_async(afqmc_ctx* ctx, double* sums_host);

/* QR stabilisation of every walker: psi^s = Q R with diag(R) > 0, psi^s <- Q,
 * log O -= sum log R_ii (all binary64). */
afqmc_status afqmc_reortho(afqmc_ctx* ctx);

/* Comb population control: ordered prefix of the weights, one uniform xi
 * (Philox stream 1, counter = the step), teeth ((k + xi) W_tot) / W, copies in
 * ascending walker order, all weights <- W_tot / W. */
afqmc_status afqmc_popcontrol(afqmc_ctx* ctx);

/* The driver loop on the device: for each of nsteps steps, the energy when
 * step % energy_every == 0 (energy_every <= 0: never), one propagation step,
 * then QR when the new step count is a multiple of reortho_every and the comb
 * when it is a multiple of comb_every (<= 0: never).  energies (host, may be
 * NULL) receives 4 sums per measurement in order; nmeas (may be NULL) their
 * count.  One synchronisation at the end. */
afqmc_status afqmc_run(afqmc_ctx* ctx, int32_t nsteps, int32_t energy_every, int32_t reortho_every,
                       int32_t comb_every, double* energies, int32_t* nmeas);

/* As afqmc_run, without synchronising: every measurement's four sums are copied to
 * energies_host + 4 k (k = 0, 1, ... in order) by an asynchronous copy enqueued right after its
 * step (with CUDA graphs on a private copy stream, so the next step does not wait for the copy;
 * the context's stream waits for the copies before the call returns: work enqueued on it later is
 * ordered after them).  Use page-locked memory for the copies to overlap; energies_host must hold 4
 * sums per measurement, and may be NULL only when energy_every <= 0.  The values are there once
 * the stream has reached the end of the call (afqmc_synchronize or any stream synchronisation).  nmeas (may be NULL)
 * receives the number of measurements at once.  Device-side conditions are reported by the next
 * synchronising call. */
afqmc_status afqmc_run_async(afqmc_ctx* ctx, int32_t nsteps, int32_t energy_every, int32_t reortho_every,
                             int32_t comb_every, double* energies_host, int32_t* nmeas);

/* Walker state (checkpoint / resume; bit-exact resume since the fields are
 * counter-based).  psi [nwalkers][norb][nalpha+nbeta][2] complex, logO
 * [nwalkers][2], w [nwalkers], step.  Any output may be NULL.  For a
 * restricted context afqmc_set_walkers requires identical alpha and beta blocks. */
afqmc_status afqmc_get_walkers(afqmc_ctx* ctx, double* psi, double* logO, double* w, uint64_t* step);
afqmc_status afqmc_set_walkers(afqmc_ctx* ctx, const double* psi, const double* w, uint64_t step);

/* Fields of the most recent propagation step: x [nwalkers][naux] and the force
 * bias shift xbar [nwalkers][naux][2] (either may be NULL). */
afqmc_status afqmc_get_fields(afqmc_ctx* ctx, double* x, double* xbar);

/* Standalone field draw: out[w][gamma] ~ N(0,1) for walker slots w < nwalkers,
 * gamma < naux, from Philox4x32-10 with key = seed and counter
 * (gamma / 2, w, step mod 2^32, (step >> 32) mod 2^16 | stream_id << 16),
 * Box-Muller with series log / sin / cos (bit-reproducible).  out: device,
 * nwalkers * naux doubles.  stream: cudaStream_t or NULL. */
afqmc_status afqmc_draw_normals(uint64_t seed, uint64_t step, uint32_t stream_id, int32_t nwalkers,
                                int32_t naux, double* out, void* stream);

afqmc_status afqmc_get_info(afqmc_ctx* ctx, afqmc_info* info);

/* Learned control variate for the exchange energy (the mixed estimator of Eq. 9 split
 * as E_L = A - K, A = Re(E0 + E1 + J) for every walker, K = the exchange term).  An MLP
 * f(z): 2 norb + 8 -> 256 -> 256 -> 256 -> 1 (tanh) of per-walker features z = [diag Re
 * G^alpha, diag Re G^beta, mean / variance / skewness / kurtosis of Re and Im vbias]
 * predicts K; exact K on m = round(sample_frac W) walkers drawn uniformly without
 * replacement each measurement (Philox stream 2) keeps the estimator unbiased:
 *   ENumer = sum_i w_i (A_i - f_i) - (W / m) sum_{i in S} w_i (K_i - f_i),
 * EDenom = sum w, E1Body = sum w Re(E0 + E1), E2Body = ENumer - E1Body.
 * The network is trained on the GPU (Adam, MSE) on (z, K) pairs the method generates.
 * cv_attach carves the network, optimiser state and a training set of `capacity` pairs
 * from a caller device block (256-byte aligned, afqmc_cv_workspace_size bytes).
 * Requires nwalkers <= 8192.  While enabled, afqmc_local_energy returns the sums only. */
afqmc_status afqmc_cv_workspace_size(afqmc_ctx* ctx, int32_t capacity, int32_t batch, size_t* bytes);
afqmc_status afqmc_cv_attach(afqmc_ctx* ctx, int32_t capacity, int32_t batch, double sample_frac, uint64_t init_seed,
                             void* dev, size_t bytes);
/* Runs nsteps plain steps (energy every step, QR / comb at the given cadences), storing every
 * walker's (z, exact K) until the training set is full; *npairs = pairs stored so far. */
afqmc_status afqmc_cv_collect(afqmc_ctx* ctx, int32_t nsteps, int32_t reortho_every, int32_t comb_every,
                              int32_t* npairs);
/* Standardises the training set (first call) and runs `epochs` of minibatch Adam; losses[e]
 * (host, may be NULL) = mean minibatch loss of epoch e (standardised units). */
afqmc_status afqmc_cv_train(afqmc_ctx* ctx, int32_t epochs, double lr, double* losses);
afqmc_status afqmc_cv_enable(afqmc_ctx* ctx, int32_t enable);
/* Network parameters [W1 (in x 256), b1, W2, b2, W3, b3, W4 (256 x 1), b4] as float32 (get: set = 0). */
afqmc_status afqmc_cv_params(afqmc_ctx* ctx, int32_t set, float* host);
/* Forward pass on rows of x [rows][dim] (network inputs); with y, also the MSE loss and every
 * gradient (same layout as the parameters).  rows <= batch. */
afqmc_status afqmc_cv_eval(afqmc_ctx* ctx, const float* x, const float* y, int32_t rows, float* out, float* loss,
                           float* grads);
afqmc_status afqmc_cv_info(afqmc_ctx* ctx, int32_t* dim, uint64_t* nparams, int32_t* npairs, int32_t* nsample);

/* Project autotuner: times `steps` propagation + energy steps of every candidate setting
 * (CUDA-core GEMM block tile 64 / 32, tensor-core, fused CUDA-core or batched-GEMM propagation and
 * the fused kernel's register tile, 1 to 4 tensor-core exchange epilogue warpgroups and the
 * exchange form) on the context's own walkers, restores the walkers,
 * keeps the fastest.
 * chosen (may be NULL) receives it; afqmc_set_tuning applies a setting directly. */
typedef struct {
  int32_t tile_cap;       /* 4: 64-wide CUDA-core GEMM tiles allowed, 2: at most 32, 1: 16 */
  int32_t prop_path;      /* propagation: 0 tensor cores in the BF16 forms (N <= 128), else the fused
                             CUDA-core kernel where it fits, else batched GEMMs; 1 batched GEMMs;
                             2 fused CUDA-core kernel */
  int32_t exch_groups;    /* tensor-core exchange epilogue warpgroups (0: largest that fits) */
  int32_t prop_tile;      /* fused propagation register tile: 0: 4 rows x 2 columns, 1: 8 x 2, 2: 4 x 4 */
  int32_t exch_form;      /* tensor-core exchange: 0 the rotated Cholesky tile resident in tensor memory
                             where it fits (BF16x3, n <= 32), else streamed; 1 both operands streamed */
  float ms_per_step;      /* measured by afqmc_autotune */
} afqmc_tuning;
afqmc_status afqmc_autotune(afqmc_ctx* ctx, int32_t steps, afqmc_tuning* chosen);
afqmc_status afqmc_set_tuning(afqmc_ctx* ctx, const afqmc_tuning* t);

/* Batched independent systems: the contexts (same device) advance in lockstep, each step being ONE
 * CUDA graph launch.  energies (host, may be NULL): [nsys][nmeas][4].  The batch launches on the
 * first context's stream; do not use the contexts concurrently.  Two forms:
 *   AFQMC_BATCH_GROUPED: every stage of the step is ONE kernel launch over the work of all systems:
 *     the exchange (with the force bias and the step's normals) and the VHS build as persistent
 *     tcgen05 kernels over a (system, spin block, tile) work list ordered by tile cost, with each
 *     system's tensor maps and parameters in device memory; the propagation as one launch over every
 *     walker of the N <= 128 systems (contiguous walker ranges per CTA balanced by cost) and one
 *     launch per Taylor product over every (walker, row tile) of the N > 128 systems; the overlap,
 *     fields, energy, QR and comb kernels as one launch over every walker.  Needs every context in
 *     the same tensor-core form (BF16 / BF16X3), real, phaseless, with the tensor-core propagation
 *     and the same Taylor order.  exch_groups caps the exchange's epilogue warpgroups (0: each
 *     system's own tuned count).  branches (0: 2, at most 4): the systems split into that many
 *     branches of about equal work, whose grouped launches run side by side on as many streams (one
 *     launch per stage and branch), so one branch's last wave overlaps another's work.  The descriptors (a few KB of device memory) are allocated on the
 *     first grouped run, not inside the caller's workspaces.
 *   AFQMC_BATCH_GRAPHS: one graph launch whose branches are the systems' own step graphs (any form).
 *   AFQMC_BATCH_AUTO (default): grouped where the contexts allow it, else graphs.
 * The graphs form gives bit for bit the results of running each context alone.  The grouped form
 * runs the same arithmetic but for the exchange, which it takes in the streamed form (both operands
 * through the shared-memory ring) at every step, also to form the force bias of steps without an
 * energy measurement: its results agree with the solo runs to the form's rounding. */
typedef struct afqmc_batch afqmc_batch;
#define AFQMC_BATCH_AUTO 0
#define AFQMC_BATCH_GROUPED 1
#define AFQMC_BATCH_GRAPHS 2
afqmc_status afqmc_batch_create(int32_t nsys, afqmc_ctx* const* ctxs, afqmc_batch** out);
afqmc_status afqmc_batch_run(afqmc_batch* b, int32_t nsteps, int32_t energy_every, int32_t reortho_every,
                             int32_t comb_every, double* energies, int32_t* nmeas);
afqmc_status afqmc_batch_set_mode(afqmc_batch* b, int32_t mode, int32_t exch_groups, int32_t branches);
/* The form the next afqmc_batch_run takes (AFQMC_BATCH_GROUPED or AFQMC_BATCH_GRAPHS). */
afqmc_status afqmc_batch_get_mode(afqmc_batch* b, int32_t* mode);
/* Stage tracing of the grouped form: with enable = 1 (counters cleared) afqmc_batch_run launches each
 * grouped stage directly between CUDA events instead of replaying its graph; afqmc_batch_stage_times
 * synchronises and returns per stage (AFQMC_STAGE_*) the milliseconds and launches so far, the
 * exchange stage being the grouped exchange kernel alone (the cleared vbias and the Theta operands
 * count as AFQMC_STAGE_FORCE_BIAS).  Either array may be NULL. */
afqmc_status afqmc_batch_profile(afqmc_batch* b, int32_t enable);
/* A text description of the grouped launches (one line per launch: problems, tiles, grid, ring
 * stages, epilogue groups, shared and tensor memory), NUL-terminated and cut to len bytes. */
afqmc_status afqmc_batch_describe(afqmc_batch* b, char* buf, size_t len);
afqmc_status afqmc_batch_stage_times(afqmc_batch* b, double* ms, int64_t* count);
void afqmc_batch_destroy(afqmc_batch* b);

/* afqmc_run replays each step pattern (energy + propagation, propagation alone, QR, comb) as a
 * CUDA graph captured on first use (enable = 1, the default); enable = 0 launches every kernel
 * directly.  Results are identical either way.  Tracing (afqmc_profile) uses direct launches. */
afqmc_status afqmc_set_graphs(afqmc_ctx* ctx, int32_t enable);
afqmc_status afqmc_set_etrial(afqmc_ctx* ctx, double e_trial);
/* E_T of the weight factor exp(dt (E_T - E_c)) (Eqs. 13-16; the paper leaves the constant out)
 * follows the estimate (enable = 1): E_T starts from its current value and two running sums from
 * zero; every energy that afqmc_run, afqmc_run_async or afqmc_batch_run measures adds its ENumer
 * and EDenom to the sums, and every comb sets E_T = sum ENumer / sum EDenom (E_T stays while the
 * sum of EDenom is 0).  The factor is common to all weights, so energies and comb decisions are
 * those of a fixed E_T; it keeps the total weight from drifting as exp(dt (E_T - E) t).  E_T then
 * lives in device memory: afqmc_get_info synchronises the stream and reports it, afqmc_set_etrial
 * overwrites it (the sums stay).  enable = 0 keeps the value reached; enabling again restarts the
 * sums.  afqmc_local_energy and free projection leave the sums alone.  Synchronises the stream. */
afqmc_status afqmc_set_etrial_update(afqmc_ctx* ctx, int32_t enable);

/* Free-projection AFQMC (Section "Free projection AFQMC"): enable = 1 switches the context to
 * unconstrained propagation.  Each step draws the fields x ~ N(0,1) with no force-bias shift
 * (xbar = 0; the mean-field subtraction and c_mf = i sqrt(dt) x.lbar stay) and carries complex
 * weights w e^{i phi}, updated by the whole overlap ratio:
 *   w e^{i phi} <- w e^{i phi} (O'/O) e^{c_mf} e^{dt (E_T - E_c)}   (no phaseless projection).
 * While enabled the four estimator sums of afqmc_local_energy, afqmc_local_energy_async and
 * afqmc_run are {Re, Im of sum w e^{i phi} E_L, Re, Im of sum w e^{i phi}} (the energy is the real
 * part of their ratio), afqmc_popcontrol and comb_every > 0 return AFQMC_EINVAL, and the control
 * variate cannot be enabled.  Switching (either way) sets every phase to 0; afqmc_set_walkers
 * does too.  The weight magnitudes w stay where afqmc_get_walkers reports them. */
afqmc_status afqmc_set_free_projection(afqmc_ctx* ctx, int32_t enable);
/* Weight phases phi [nwalkers] (host, radians in (-pi, pi]); all 0 in phaseless propagation. */
afqmc_status afqmc_get_weight_phases(afqmc_ctx* ctx, double* phase);

/* Wait for the context's stream, polling, for at most timeout_s seconds. */
afqmc_status afqmc_synchronize(afqmc_ctx* ctx, double timeout_s);

/* Free host-side state (the caller frees the workspace afterwards). */
void afqmc_destroy(afqmc_ctx* ctx);

/* Tracing: per-stage device time from CUDA events recorded on the context's
 * stream around each stage.  enable = 1 resets the counters and starts
 * recording, 0 stops.  afqmc_stage_times synchronises the stream and returns,
 * for each of the AFQMC_NSTAGES stages, the accumulated milliseconds and the
 * number of timed stage executions (either output may be NULL). */
enum {
  AFQMC_STAGE_OVERLAP = 0,     /* overlap, LU, log det, Theta (+ weight update) */
  AFQMC_STAGE_FORCE_BIAS = 1,  /* vbias when the energy was not measured at the same walkers */
  AFQMC_STAGE_EXCHANGE = 2,    /* T = Ltilde Theta contraction: exchange partials + vbias */
  AFQMC_STAGE_ENERGY = 3,      /* per-walker E_L assembly and the weighted sums */
  AFQMC_STAGE_FIELDS = 4,      /* Philox fields, shift, VHS coefficients */
  AFQMC_STAGE_VHS = 5,         /* VHS = sum_g coef_g L^g */
  AFQMC_STAGE_PROPAGATE = 6,   /* exp(-dt/2 h_eff) Taylor(VHS) exp(-dt/2 h_eff) on the walkers */
  AFQMC_STAGE_QR = 7,
  AFQMC_STAGE_COMB = 8,
  AFQMC_NSTAGES = 9
};
afqmc_status afqmc_profile(afqmc_ctx* ctx, int32_t enable);
afqmc_status afqmc_stage_times(afqmc_ctx* ctx, double* ms, int64_t* count);

/* Number of kernel launches the context has issued (for launch accounting). */
uint64_t afqmc_launch_count(afqmc_ctx* ctx);

const char* afqmc_last_error(void);

/* Comb population-control plan that allocates nothing.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory: callers whose device memory is owned entirely by another
 * allocator (a framework's caching pool or an arena reserved up front), and
 * callers in latency-critical loops that must not trigger the implicit
 * device-wide synchronisation of cudaMalloc/cudaFree.  It needs no context and
 * no workspace.
 *   w       device, [nwalkers] binary64 walker weights, each finite and >= 0 (input)
 *   src     device, [nwalkers] int32: source walker of every new slot (output)
 *   neww    device, one binary64: the common new weight W_tot / nwalkers, or
 *           -1 if the weight total W_tot is not positive and finite (every
 *           weight zero, or a NaN / Inf weight); src is then the identity
 *           (output).  neww is the only signal: the call itself returns
 *           without waiting for the kernel.
 * xi comes from Philox stream 1 at counter `step`, exactly as in
 * afqmc_popcontrol, so src and neww equal what afqmc_popcontrol applies.
 * Scratch: the prefix sums live in a file-scope device array of
 * AFQMC_NOALLOC_MAX_WALKERS + 64 eight-byte words (about 513 KiB) that every
 * GPU which loads the library holds until the process exits; nwalkers above
 * AFQMC_NOALLOC_MAX_WALKERS is rejected with AFQMC_EINVAL.  Set-up: the first
 * call on a device (and the first after that device's context was destroyed
 * and created again) looks the array's address up (cudaGetSymbolAddress) with
 * that device current.  That first lookup may itself create the CUDA context
 * and load the library's device code (lazy module loading), which reserves
 * device memory and may synchronise; so make the first call outside any
 * latency-critical loop and before any stream capture.  Later calls only
 * enqueue.  Every call shares the one array and overwrites it: calls whose
 * kernels can overlap on the GPU (other streams, other host threads) race and
 * may return wrong plans, so order them on one stream.  Enqueued on `stream`
 * (NULL: default stream); returns without synchronising.  No cudaMalloc,
 * cudaFree or allocating library routine is called. */
#define AFQMC_NOALLOC_MAX_WALKERS 65536
afqmc_status afqmc_comb_plan_noalloc(const double* w, int32_t nwalkers, uint64_t seed, uint64_t step,
                                     int32_t* src, double* neww, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AFQMC_H */
