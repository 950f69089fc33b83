/*
 * epw.h -- C ABI of the GB300 (sm_103a) electron-linewidth library.
 *
 * The library evaluates the hot path of EPW's method (Ponce, Margine, Verdi,
 * Giustino, Comput. Phys. Commun. 209, 116 (2016)):
 *
 *   Wannier interpolation of the electronic Hamiltonian H(Re), the force
 *   constants Phi(R) and the electron-phonon vertex g(Re,Rp) onto lists of
 *   k and q points (the "standard Wannier electron-phonon interpolation",
 *   step (iii) of Sec. "Electron-phonon coupling in polar materials"), the
 *   rotation of g into the Bloch / phonon-mode basis with the U matrices of
 *   the interpolated Hamiltonian (overlap equation of the same section), and
 *   the electron linewidth of Eq. (linewidthel):
 *
 *     Im Sigma_nk = pi sum_{m,nu} sum_q w_q |g_mn,nu(k,q)|^2
 *        { [n_qnu + f_mk+q] delta(e_nk - e_mk+q + w_qnu)
 *        + [n_qnu + 1 - f_mk+q] delta(e_nk - e_mk+q - w_qnu) }
 *
 *   evaluated on shell (w = e_nk - e_F, Sec. "Examples": Sigma''(e_nk)), with
 *   Bose-Einstein n and Fermi-Dirac f (definitions after Eq. phselfenergy) and
 *   a Gaussian delta(x) = exp(-(x/sigma)^2) / (sigma sqrt(pi)).  1/tau = 2 Im
 *   Sigma (Eq. scatteringRate) is left to the caller.
 *
 * Conventions
 *   - k, q and R are in crystal coordinates; R are integer triples.  Phases
 *     are e^{+2 pi i x.R}; the argument x.R is reduced modulo 1 in FP64.
 *       H(k)     = sum_Re wRe e^{2pi i k.Re} H(Re)
 *       D(q)     = sum_R  wR  e^{2pi i q.R} Phi(R) / sqrt(M_kappa M_kappa')
 *       g(k,q)   = sum_Re sum_Rp wRe wRp e^{2pi i (k.Re + q.Rp)} g(Re,Rp)
 *       g_mn,nu  = sum_{kappa alpha} [U_k+q^+ g_{kappa alpha}(k,q) U_k]_mn
 *                    e_{kappa alpha,nu}(q) / sqrt(2 M_kappa w_qnu)
 *     with H(k) U_k = U_k diag(e_k) (eigenvalues ascending) and
 *     D(q) e_nu = w_nu^2 e_nu, w_nu = sign(w^2) sqrt|w^2|.  Modes with
 *     w_qnu < omega_min are left out of every sum.
 *   - Energies in eV, temperatures in K, k_B = 8.617333262e-5 eV/K.
 *   - Complex arrays are interleaved (re, im) doubles, row-major, C order.
 *
 * Pointers
 *   - epw_wannier_desc arrays are HOST pointers; the model copies them.
 *   - k, q, wq and every output may be host or device pointers; the library
 *     tells them apart with cudaPointerGetAttributes.  With device pointers a
 *     call is asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 *     stream); with any host pointer the call stages through device memory and
 *     returns after the results are copied back.
 *   - Outputs are caller-owned.  The model owns its device buffers and a
 *     workspace that grows on demand (epw_reserve pre-sizes it).
 *
 * Errors
 *   Every entry point returns an epw_status; on failure outputs are undefined,
 *   nothing is freed and epw_last_error() returns a message (per thread).
 *   Device-side failures (an eigensolver that did not converge within its sweep
 *   cap) raise a flag that epw_sync() reports; calls with host outputs check it
 *   before returning.  No exception crosses the ABI.
 */
#ifndef EPW_H
#define EPW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EPW_ABI_VERSION 1
#define EPW_MAX_NW 18    /* largest number of Wannier functions */
#define EPW_MAX_MODES 18 /* largest 3*nat */

typedef enum {
  EPW_OK = 0,
  EPW_ERR_INVALID_ARG = 1,
  EPW_ERR_CUDA = 2,
  EPW_ERR_OOM = 3,
  EPW_ERR_NOT_CONVERGED = 4,
  EPW_ERR_TIMEOUT = 5,
  EPW_ERR_UNSUPPORTED = 6
} epw_status;

/* Arithmetic of the interpolation contractions and the per-pair eigensolves.
 *   EPW_FP64   : everything in FP64 (CUDA cores).
 *   EPW_FP32   : contractions, eigensolves and rotations in FP32 (CUDA cores);
 *                phases, phonons, k-side eigensolves and the reduction in FP64.
 *   EPW_BF16X3 : contractions on the tensor cores (tcgen05) with operands split
 *                into two bfloat16 terms (x = hi + lo; hi*hi + hi*lo + lo*hi,
 *                FP32 accumulation); per-pair eigensolves and rotations in
 *                FP32; phases, phonons, k-side work and the reduction in FP64.
 *   EPW_TF32X3 : as EPW_BF16X3 with tf32 terms (about 16x smaller contraction
 *                error, half the tensor throughput).
 * The split forms serve every shape up to nw = 18, 3nat = 18 with Re and Rp
 * equal or not (the contraction runs over both sets); the entry points that
 * have per-pair kernels only up to nw = 8, 3nat = 9 (adjoint, phonon-side sums,
 * complex self-energy) say so and return EPW_ERR_UNSUPPORTED beyond. */
typedef enum { EPW_FP64 = 0, EPW_FP32 = 1, EPW_BF16X3 = 2, EPW_TF32X3 = 3 } epw_precision;

typedef struct epw_model epw_model; /* opaque */

/* Real-space inputs (HOST pointers).  Weights may be NULL (all ones).
 *   mass [nat]
 *   Re  [nRe][3]  int32,  wRe  [nRe],  H   [nRe][nw][nw] complex
 *   Rph [nRph][3] int32,  wRph [nRph], Phi [nRph][3nat][3nat] complex,
 *        row/column index kappa*3 + alpha
 *   Rp  [nRp][3]  int32,  wRp  [nRp],  g   [nRe][nRp][3nat][nw][nw] complex
 *        (g_{kappa alpha}(Re,Rp)_{mn}); complex128 unless g_is_c64 != 0, in
 *        which case g holds interleaved float pairs. */
typedef struct {
  int nw, nat;
  const double *mass;
  int nRe;
  const int32_t *Re;
  const double *wRe;
  const double *H;
  int nRph;
  const int32_t *Rph;
  const double *wRph;
  const double *Phi;
  int nRp;
  const int32_t *Rp;
  const double *wRp;
  const void *g;
  int g_is_c64;
} epw_wannier_desc;

typedef struct {
  double T_K;          /* temperature (K), >= 0 */
  double EF_eV;        /* Fermi level (eV) */
  double sigma_eV;     /* Gaussian width (eV), > 0 */
  double omega_min_eV; /* modes below this frequency are left out (eV), >= 0 */
  int precision;       /* epw_precision */
  int reserved;        /* must be 0 */
} epw_params;

/* Copy a Wannier model onto the current CUDA device.  Returns EPW_ERR_INVALID_ARG
 * for sizes outside 1 <= nw <= EPW_MAX_NW, 1 <= 3*nat <= EPW_MAX_MODES, empty R
 * sets, or a non-positive mass; EPW_ERR_OOM when device memory runs out. */
epw_status epw_load_wannier(const epw_wannier_desc *desc, epw_model **out);

/* Replace the vertex g(Re,Rp) of a loaded model (same layout and sizes as in
 * epw_wannier_desc; weights are applied as at load).  g may be a host or a
 * device pointer; complex128 unless g_is_c64.  Stream-ordered on `stream`:
 * later calls on the same stream see the new vertex.  Used for gradient
 * descent on g with epw_linewidth_backward. */
epw_status epw_set_vertex(epw_model *model, const void *g, int g_is_c64, void *stream);

/* Release a model and its device memory (NULL is a no-op).  Not stream-ordered:
 * the caller makes sure no work that uses the model is still running. */
void epw_free_model(epw_model *model);

/* Pre-size the workspace for calls with up to nk k-points and nq q-points at
 * the given precision (so that later calls do not allocate, e.g. inside a CUDA
 * graph capture). */
epw_status epw_reserve(epw_model *model, int nk, int nq, int precision);

/* Planning without a model or a device: the device workspace (bytes) that
 * epw_linewidth, or epw_reserve, takes for a model of this shape -- nw Wannier
 * functions, nat atoms, nRe / nRp / nRph lattice vectors of H, g and the force
 * constants, same_ep / same_eph nonzero when the Re and Rp (Re and Rph) sets are
 * identical, polar nonzero with a long-range vertex -- on nk k-points and nq
 * q-points (k, q and weights as host arrays) in the given precision, and the k
 * per pass (nk when the k list runs in one pass; see EPW_K_SIDE_BYTES under
 * epw_linewidth).  The figures follow the same plan the library lays out at
 * run time, with the environment as it is at the call.  Either output may be
 * NULL.  Errors: EPW_ERR_INVALID_ARG for sizes outside the limits of
 * epw_load_wannier, unequal sizes of sets declared identical, or an unknown
 * precision; EPW_ERR_UNSUPPORTED where epw_linewidth has no form for the shape
 * in that precision.  Reads no device state and launches nothing. */
epw_status epw_plan_linewidth(int nw, int nat, int nRe, int nRp, int nRph, int same_ep, int same_eph, int polar,
                              int nk, int nq, int precision, size_t *ws_bytes, int *k_per_pass);

/* Interpolated quantities on the product k x q (the unreduced path):
 *   eps_k  [nk][nw]          band energies at k (FP64)
 *   eps_kq [nk][nq][nw]      band energies at k+q
 *   omega  [nq][3nat]        phonon frequencies
 *   g      [nk][nq][3nat][nw][nw] complex  g_mn,nu(k,q) (index order nu, m, n);
 *                            zero for modes below omega_min.
 * Any output may be NULL (not written).  Per-element g depends on the
 * eigenvector gauge inside degenerate subspaces; sums over degenerate blocks
 * do not.  nk, nq >= 0 (zero is a no-op). */
epw_status epw_interp_g(const epw_model *model, int nk, const double *k, int nq, const double *q,
                        int precision, double omega_min_eV, double *eps_k, double *eps_kq,
                        double *omega, double *g, void *stream);

/* Electron linewidth Im Sigma_nk [nk][nw] (eV) on the k list, summed over the
 * q list with weights wq (NULL: 1/nq each).  Sums of the positive terms are
 * deterministic (fixed order, compensated in FP64).
 * Split precisions run on the tensor cores: models whose per-k columns
 * 2 nw^2 (3nat + 1) fit 128 take one fused kernel (on CTA pairs, 2-SM MMAs over
 * 256 q rows; EPW_NARROW_FORM=single selects single CTAs); (nw, 3nat) = (8, 6) and
 * (5, 9) take the wide-shape form (H(k+q) eigensolve beside the vertex
 * contraction; only terms whose Gaussians do not underflow in FP32 are
 * evaluated, which leaves the sums unchanged), whose fused kernel runs on CTA
 * pairs (2-SM MMAs over 256 q rows; the environment variable EPW_WIDE_FORM=single
 * selects the single-CTA kernel, EPW_WIDE_FORM=split a two-kernel variant);
 * other shapes take the staged form (the contraction per chunk of k on the
 * tensor cores, then one warp per pair; for nw > 8 or 3nat > 9 that warp
 * evaluates only the terms within the same cutoff, EPW_STAGED_PAIR=dense every
 * term).  When the buffers that grow with nk (bands and vertex at k, operands,
 * partial sums; a staged contraction chunk counts once, at its capped size)
 * would exceed EPW_K_SIDE_BYTES (environment; 8 GiB by default), the k list
 * runs in equal passes, each with the whole q list (results do not depend on
 * the pass count). */
epw_status epw_linewidth(const epw_model *model, int nk, const double *k, int nq, const double *q,
                         const double *wq, const epw_params *params, double *imsigma, void *stream);

/* Adjoint of L = sum_{k,n} grad_imsigma[k][n] * Im Sigma_nk:
 *   dg  [nRe][nRp][3nat][nw][nw] complex: dL/dRe g + i dL/dIm g  (may be NULL)
 *   dT, dEF: dL/dT and dL/dE_F (host or device double, may be NULL).
 * g(k,q) is recomputed, not stored.  Requires T_K > 0. */
epw_status epw_linewidth_backward(const epw_model *model, int nk, const double *k, int nq,
                                  const double *q, const double *wq, const epw_params *params,
                                  const double *grad_imsigma, double *dg, double *dT, double *dEF,
                                  void *stream);

/* Phonon-side sums over a k list of the same interpolated vertex, for each q
 * of the q list and each mode nu (Sec. "Theory", Eqs. (linewidthph),
 * (lambdaEQ), (nestingfct)):
 *   pi_imag[q][nu] = Pi''_qnu on shell (w = w_qnu), sign as printed:
 *       2 pi sum_k w_k sum_mn |g_mn,nu(k,q)|^2 (f_nk - f_mk+q) delta(e_nk - e_mk+q - w_qnu)
 *   lambda[q][nu]  = sum_k w_k sum_mn |g|^2 delta(e_nk - E_F) delta(e_mk+q - E_F) / (N(E_F) w_qnu)
 *   nesting[q]     = sum_k w_k sum_mn delta(e_nk - E_F) delta(e_mk+q - E_F)
 *   dos_ef[0]      = N(E_F) = sum_k w_k sum_n delta(e_nk - E_F)   (per spin)
 * with the Gaussian delta and occupations of epw_linewidth (params: T_K,
 * EF_eV, sigma_eV, omega_min_eV; modes below omega_min get 0).  k [nk][3],
 * wk [nk] or NULL (1/nk), q [nq][3]; outputs [nq][3nat], [nq][3nat], [nq], [1]
 * (eV for pi_imag; lambda and nesting dimensionless / per eV^2); any output may
 * be NULL; pointers host or device.  precision: EPW_FP64, EPW_FP32 (CUDA
 * cores) or EPW_TF32X3 / EPW_BF16X3 (contraction on the tensor cores, staged
 * per chunk of k).  Shapes up to nw = 8, 3nat = 9; others
 * return EPW_ERR_UNSUPPORTED.  Per-q sums over k are formed in a fixed order. */
epw_status epw_phonon_selfenergy(const epw_model *model, int nk, const double *k, const double *wk, int nq,
                                 const double *q, const epw_params *params, double *pi_imag, double *lambda,
                                 double *nesting, double *dos_ef, void *stream);

/* Complex electron self-energy of Eq. (elselfenergy) on a frequency grid, with
 * the broadening i delta (delta > 0, eV) and omega measured from E_F:
 *   sigma[k][n][i] = sum_q w_q sum_{m,nu} |g_mn,nu(k,q)|^2
 *        [ (n_qnu + f_mk+q) / (omega_i - (e_mk+q - E_F) + w_qnu + i delta)
 *        + (n_qnu + 1 - f_mk+q) / (omega_i - (e_mk+q - E_F) - w_qnu + i delta) ]
 * (complex, re/im interleaved, [nk][nw][nomega]), and, when spectral != NULL, the
 * spectral function of Eq. (spectral_funct)
 *   spectral[k][n][i] = (1/pi) |Sigma''| / ((omega_i - (e_nk - E_F) - Sigma~'(omega_i))^2 + Sigma''^2),
 * Sigma'' = -Im Sigma, Sigma~' = Re Sigma(omega) - Re Sigma(0) (Eq. realpartselfenergy).
 * params: T_K, EF_eV, omega_min_eV and precision as for epw_linewidth (sigma_eV is not
 * used: the width here is delta).  Host or device pointers.  FP64/FP32 on the CUDA cores,
 * TF32X3/BF16X3 with the contraction staged on the tensor cores.  Shapes up to
 * nw = 8, 3nat = 9.  Sums over q in a fixed order. */
epw_status epw_selfenergy(const epw_model *model, int nk, const double *k, int nq, const double *q,
                          const double *wq, const epw_params *params, double delta, int nomega,
                          const double *omega, double *sigma, double *spectral, void *stream);

/* Isotropic Eliashberg function of Eq. (isotropiceliash) on an omega grid:
 *   a2f[i] = 1/2 sum_q w_q sum_nu omega[q][nu] lambda[q][nu] delta_ph(grid[i] - omega[q][nu])
 * with delta_ph the Gaussian exp(-(x/sigma_ph)^2)/(sigma_ph sqrt(pi)); omega and lambda [nq][nmodes]
 * (from epw_interp_g and epw_phonon_selfenergy), wq [nq] or NULL (1/nq), grid [ngrid] (eV) and
 * a2f [ngrid] (dimensionless).  Host or device pointers; host inputs are staged through
 * stream-ordered scratch of the call, and a host a2f is ready on return.
 * Each grid point is a compensated sum over (q, nu) in a fixed order. */
epw_status epw_eliashberg(int nq, int nmodes, const double *omega, const double *lambda, const double *wq,
                          int ngrid, const double *grid, double sigma_ph, double *a2f, void *stream);

/* Allocation-free variant of epw_linewidth, for callers that cannot allocate
 * device memory: code running where cudaMalloc is not allowed or not wanted
 * (inside a memory-pool-managed host framework, a real-time loop that must
 * not block on the allocator, a sandbox that forbids new device allocations).
 * The paper has no counterpart; it is an integration convenience.
 *   - No device memory is allocated or freed by this call (no cudaMalloc,
 *     cudaFree or allocating library routine).  Its scratch is one fixed
 *     device array of EPW_NOALLOC_SCRATCH_BYTES that the library holds on every
 *     GPU where it is loaded until the process exits.  Problems whose scratch
 *     exceeds it return EPW_ERR_INVALID_ARG with the bytes needed.
 *   - The model must already be loaded (epw_load_wannier allocates).
 *   - k, q, wq (or NULL) and imsigma must be device pointers; precision
 *     EPW_FP64 or EPW_FP32.  The call is asynchronous on `stream`; device-side
 *     failures are reported by epw_sync.
 *   - The first call on a device looks up the scratch array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the one array, which keeps the last call's contents
 *     (every value a call reads it first writes).  Calls whose work overlaps
 *     on the GPU (different streams, threads or processes sharing a context)
 *     race on it: serialise them. */
#define EPW_NOALLOC_SCRATCH_BYTES (32u << 20)
epw_status epw_linewidth_noalloc(const epw_model *model, int nk, const double *k, int nq, const double *q,
                                 const double *wq, const epw_params *params, double *imsigma, void *stream);

/* ---------------------------------------------------------------- batches
 * Many linewidth problems of Eq. (linewidthel) at once, on systems that may
 * differ in every size (nw, nat, nRe, nRp, nk, nq), precision and parameter.
 * One job is one epw_linewidth call; all its pointers are DEVICE pointers:
 *   k [nk][3], q [nq][3], wq [nq] or NULL (1/nq), imsigma [nk][nw] (output).
 * Several jobs may share a model.  Shapes, pointers and params are fixed when
 * the batch is created; the contents of k, q and wq may change between runs. */
typedef struct {
  const epw_model *model;
  int nk, nq;
  const double *k, *q, *wq;
  epw_params params;
  double *imsigma;
} epw_linewidth_job;

typedef struct epw_batch epw_batch;

/* Plans the jobs and allocates one device workspace for all of them (owned by
 * the batch; four regions, each as large as the largest job of the jobs that
 * share it and run one after another), picks each job's tile parameters with
 * the autotuner, and
 * captures the whole batch as one CUDA graph whose jobs run on parallel
 * branches (the branch count is chosen by timing the candidate graphs; a batch
 * whose first pass takes over 5 s takes four branches without timing).
 * Jobs whose buffers would grow past EPW_K_SIDE_BYTES (environment; 8 GiB by
 * default) with their k count run their k list in passes, as epw_linewidth does.
 * Autotuning runs timed trials of a job shape the first time the process
 * sees it (kept per process; with the environment variable EPW_TUNE_CACHE
 * naming a file, also read from and appended to it).  Creating a batch runs
 * every job at least once, so each imsigma holds a result on return.
 * Errors: EPW_ERR_INVALID_ARG (null/host pointers, bad params, models on
 * another device), EPW_ERR_UNSUPPORTED (a job shape with no kernel for its
 * precision), EPW_ERR_OOM, EPW_ERR_CUDA.  No model may have timing enabled. */
epw_status epw_batch_create(int njobs, const epw_linewidth_job *jobs, epw_batch **out);
/* Replays the batch's graph on `stream` (asynchronous); epw_sync on a job's
 * model reports device-side failures. */
epw_status epw_batch_run(epw_batch *batch, void *stream);
/* Graph branches, workspace bytes and the number of kernel nodes of the graph (the
 * kernels one replay launches); any output may be NULL. */
epw_status epw_batch_info(const epw_batch *batch, int *branches, size_t *workspace_bytes, size_t *graph_nodes);
/* Waits for the batch's work and releases its graph, streams and workspace. */
void epw_batch_free(epw_batch *batch);
/* One-shot form: create, run on `stream`, wait, check every model's device
 * status, free. */
epw_status epw_linewidth_batched(int njobs, const epw_linewidth_job *jobs, void *stream);

/* Long-range (polar) part of the vertex, Sec. "Electron-phonon coupling in
 * polar materials", Eq. (long-range), with the overlap in its small-(q+G) form
 * [U_k U_k+q^dagger]_nm of that section.  Once set, every interpolated vertex of
 * the model is g = g^S + g^L with g^S the Wannier-interpolated g(Re,Rp) and
 *   g^L_mn,nu(k,q) = i C_nu(q) [U_k+q^dagger U_k]_mn,
 *   C_nu(q) = prefactor sum_{kappa,a} e_{kappa a,nu}(q) / sqrt(2 M_kappa w_qnu)
 *             sum_{G, q+G != 0} exp(-(q+G).eps.(q+G) / (4 alpha)) ((q+G).Z*_kappa)_a / ((q+G).eps.(q+G)),
 * (x.Z*)_a = sum_b x_b Z*_{kappa, b a}, q + G Cartesian from the lattice vectors A
 * (rows, any length unit L; b_i . a_j = 2 pi delta_ij), G = sum n_i b_i with
 * |n_i| <= gmax.  The printed equation has no prefactor and no convergence factor
 * for the G sum: prefactor (eV L^-1 scale of the model's vertex) and alpha (L^-2)
 * are inputs.  Zstar [nat][3][3] host memory, copied.  NULL removes the term. */
typedef struct {
  double A[3][3];
  double eps_inf[3][3];
  const double *Zstar;
  double alpha;
  double prefactor;
  int gmax;
} epw_polar_desc;
epw_status epw_set_polar(epw_model *model, const epw_polar_desc *polar);

/* Self-test of the device failure path on the current GPU: a kernel waits,
 * with the same bounded mbarrier wait the tensor-core kernels use, on a barrier
 * that nothing arrives at, for `cycles` clock cycles (1..4e9; 2e6 is about 1 ms).
 * The wait gives up, raises the device timeout flag and the kernel returns; the
 * call then returns EPW_ERR_TIMEOUT (the expected outcome) with *waited_out = 1.
 * No fault, trap or hang is involved and the context stays usable. */
epw_status epw_selftest_wait_timeout(long long cycles, int *waited_out);

/* Wait for the model's work on `stream` and report device-side failures
 * (EPW_ERR_NOT_CONVERGED) raised since the previous epw_sync; clears them. */
epw_status epw_sync(const epw_model *model, void *stream);

/* Model sizes: nw, nat, nRe, nRp, nRph (any pointer may be NULL). */
epw_status epw_model_info(const epw_model *model, int *nw, int *nat, int *nRe, int *nRp, int *nRph);

/* Number of kernel launches the library has issued in this process. */
uint64_t epw_launch_count(void);

/* Measurement hook.  While enabled, each launch of the dominant (per-pair)
 * kernel is bracketed by CUDA events recorded on its launch stream (at most
 * 4096 launches are kept); the wide-shape tensor-core form also brackets its
 * per-pair eigensolve kernel, as a second tag.  epw_timing_read synchronizes
 * those events and returns the summed device time (ms) and the number of
 * launches of the dominant kernel, then clears them all.
 * epw_timing_read_tags returns both tags: ms2[0], n2[0] the dominant kernel,
 * ms2[1], n2[1] the secondary one (either pointer may be NULL), then clears. */
epw_status epw_timing_enable(epw_model *model, int enable);
epw_status epw_timing_read(epw_model *model, double *total_ms, int *launches);
epw_status epw_timing_read_tags(epw_model *model, double *ms2, int *n2);

/* Message of the last failed call on this thread ("" if none). */
const char *epw_last_error(void);

/* EPW_ABI_VERSION of the loaded library. */
int epw_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EPW_H */
