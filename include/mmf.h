/*
 * mmf.h -- C ABI of the GB300 multimode Floquet library (libmmf.so).
 *
 * Problem (arXiv 2005.03426, Eq. 1): a D-level system with static Hamiltonian H0 driven at
 * K incommensurate frequencies omega_l,
 *     H(t) = H0 + sum_{l,h} ( V^{l,h} e^{+i h omega_l t} + V^{l,h}^dagger e^{-i h omega_l t} ),
 * so a real drive A cos(omega t) O (O Hermitian) is given as V = (A/2) O at harmonic 1.
 * The library builds the Floquet matrix H_F of Eq. 6 truncated to |n_l| <= N_l
 * (n = D prod_l (2 N_l + 1), layout of Appendix A: mode 1 innermost), diagonalises it on the
 * GPU, and evaluates from its eigenpairs the time-evolution operator U(t, t0) (Eq. 3-5) and
 * the time-averaged transition probabilities Pbar_{i->j}.
 *
 * Conventions
 *   - Complex arrays are interleaved (re, im) doubles (C99 double _Complex layout).
 *   - Host pointers are owned by the caller and only read or written during the call.
 *   - Matrices given to the library (H0, V) are D x D row-major.
 *   - Every function returns an int status: MMF_OK (0), a negative MMF_ERR_* code for an
 *     invalid argument or resource problem, or a positive MMF_ST_* numerical status.
 *     mmf_strerror() gives a message; mmf_last_error() the detail of the last failure on the
 *     calling thread.
 *   - A context is bound to one CUDA device and one stream; calls on one context are
 *     serialised internally.  All GPU work of a context runs on its stream.
 *   - Nothing falls back to the CPU: without a usable GPU every call that needs one fails
 *     with MMF_ERR_CUDA.
 */
#ifndef MMF_H
#define MMF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MMF_API __attribute__((visibility("default")))
#else
#define MMF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define MMF_OK 0
#define MMF_ERR_ARG -1        /* invalid argument (null pointer, bad size, non-Hermitian H0...) */
#define MMF_ERR_STATE -2      /* call out of order (e.g. results before diagonalise) */
#define MMF_ERR_BUDGET -3     /* the request does not fit the context's HBM budget */
#define MMF_ERR_CUDA -4       /* a CUDA runtime call failed (no device, launch error...) */
#define MMF_ERR_UNSUPPORTED -5 /* size or option outside what this build supports */
#define MMF_ERR_NOMEM -6      /* host allocation failed */
#define MMF_ST_NOCONV 1       /* an iteration reached its cap (Jacobi sweeps, bisection) */
#define MMF_ST_NONFINITE 2    /* NaN or Inf met in the input or a result */
#define MMF_ST_CLUSTER 3      /* mixed refinement met a cluster of more than 32 close eigenvalues:
                                 its vectors are orthonormal but not separated inside the cluster */

/* ---------------------------------------------------------------- precision */
#define MMF_FP64 0   /* every step in FP64 */
#define MMF_MIXED 1  /* FP32 reduction + FP64 tridiagonal solve + Ogita-Aishima refinement */

typedef struct mmf_ctx mmf_ctx;
typedef struct mmf_sys mmf_sys;
typedef struct mmf_batch mmf_batch;
typedef struct mmf_server mmf_server;

/* ---------------------------------------------------------------- context
 * mmf_ctx_create: bind to CUDA device `device` and stream `cuda_stream` (a cudaStream_t, or
 * NULL for a stream the context creates and owns).  hbm_budget_bytes caps the device memory
 * all batches of this context may hold at once (0 = 90% of the device's free memory, counting
 * memory that the process's stream-ordered pool holds unused as free).
 * Errors: MMF_ERR_ARG (out == NULL), MMF_ERR_CUDA (no such device).
 */
MMF_API int mmf_ctx_create(int device, size_t hbm_budget_bytes, void* cuda_stream, mmf_ctx** out);
/* Frees the context; batches and systems created on it must be destroyed first. */
MMF_API int mmf_ctx_destroy(mmf_ctx* ctx);
/* Device bytes currently held by the context's batches. */
MMF_API size_t mmf_ctx_bytes_in_use(const mmf_ctx* ctx);
MMF_API size_t mmf_ctx_budget(const mmf_ctx* ctx);
/* Size thresholds of the solver paths for batches created afterwards (value < 0 restores the
 * default): MMF_OPT_JACOBI_N_FP64 / _MIXED: largest n solved by the shared-memory Jacobi kernel
 * (defaults 84 / 118, also the maxima; values below 4 act as 4); MMF_OPT_LARGE_N: smallest n reduced by the whole-GPU
 * Householder reduction, one system at a time (default: sizes one CTA's shared memory cannot
 * hold); MMF_OPT_REFINE_FULL_N: in the mixed path, smallest n whose second refinement step is a
 * full one (default 3000).  Below it the second step is hybrid, like the first: the corrections
 * of all pairs from C = X^H W on the tensor cores, with G = X^H X formed FP64-accurately only for
 * pairs within 16 places in the sorted order; a full step also forms all of G (costlier, for the
 * dense spectra of large H_F).
 * MMF_OPT_GRAM_KERNEL: the full second step's Gram product X^H X, 0 (default) on the BF16 tensor
 * cores by exact integer slicing, 1 in double-FP32 on the FP32 units (both FP64-accurate).
 * MMF_OPT_BT_TC_N: in the mixed path, smallest n whose back-transform (Z = Q Y, Sec. 3.2's
 * eigenvectors from the tridiagonal ones) runs on the tensor cores in split TF32 (default 256);
 * smaller systems use the FP32 SIMT kernel.
 * MMF_OPT_BAND_MAX: largest half-bandwidth b of H_F (the farthest nonzero from the diagonal, set
 * by the couplings' block offsets of Eq. 6 / Appendix A) for which a system is reduced to
 * tridiagonal form by Householder bulge chasing on its band (O(n^2 b) work) instead of the dense
 * reduction (O(n^3)); at most 64; 0 switches the band path off.  Default: 64 on the FP64 path,
 * 0 on the mixed path (whose dense reduction and tensor-core back-transform are faster at the
 * benchmark sizes).  Systems with n < 2 b + 2 use the dense reduction.
 * MMF_OPT_JACOBI_SWEEPS: iteration cap of the shared-memory Jacobi kernel (default 40 sweeps;
 * values below 1 act as 1).  A system that has not converged at the cap gets MMF_ST_NOCONV from
 * mmf_batch_sync / mmf_diagonalise.
 * MMF_OPT_HETRD_TC: in the mixed path, the dense Householder reduction's trailing update
 * A -= V W^H + W V^H after each panel (Sec. 3.2's diagonalisation) on the tensor cores in split
 * TF32 (1 or < 0, default) or on the FP32 units (0).
 * Results do not depend on the path beyond rounding. */
#define MMF_OPT_JACOBI_N_FP64 1
#define MMF_OPT_JACOBI_N_MIXED 2
#define MMF_OPT_LARGE_N 3
#define MMF_OPT_REFINE_FULL_N 4
#define MMF_OPT_GRAM_KERNEL 5
#define MMF_OPT_BT_TC_N 6
#define MMF_OPT_JACOBI_SWEEPS 7
#define MMF_OPT_BAND_MAX 8
#define MMF_OPT_HETRD_TC 9
MMF_API int mmf_ctx_set_option(mmf_ctx* ctx, int option, int64_t value);
/* Tuning rules (per-system solver choices measured by an autotuner, e.g. the package's tune.py):
 * for batches created afterwards, a system of the given precision with n_lo <= n <= n_hi and
 * half-bandwidth band_lo <= b <= band_hi (b as for MMF_OPT_BAND_MAX) takes
 *   jacobi: 1 the shared-memory Jacobi kernel (if n is within its maximum), 0 the Householder paths;
 *   band:   1 the band path (if the band allows it), 0 the dense reduction;
 *   bt_tc:  1 / 0 the mixed path's dense back-transform on the tensor cores / on the FP32 units;
 * each -1 = no preference (the size thresholds above decide).  The first matching rule wins; a
 * system's choices depend only on its own n and band, never on the rest of its batch.
 * mmf_ctx_load_tuning reads rules from a text file, one per line:
 *   <fp64|mixed> n_lo n_hi band_lo band_hi jacobi band bt_tc      ('#' starts a comment)
 * and returns the number of rules added (or a negative error with the line in mmf_last_error).
 * Results do not depend on the choices beyond rounding. */
MMF_API int mmf_ctx_add_rule(mmf_ctx* ctx, int precision, int64_t n_lo, int64_t n_hi, int band_lo, int band_hi,
                             int jacobi, int band, int bt_tc);
MMF_API int mmf_ctx_clear_rules(mmf_ctx* ctx);
MMF_API int mmf_ctx_load_tuning(mmf_ctx* ctx, const char* path);

/* ---------------------------------------------------------------- system definition
 * The paper's set-up step (Sec. 3.1: the ATOM type, the harmonics array and the MODE
 * type; Eq. 1).  H0 is D x D, Hermitian (checked to 1e-12 relative; otherwise MMF_ERR_ARG).
 */
MMF_API int mmf_sys_create(mmf_ctx* ctx, int D, const double* H0, mmf_sys** out);
/* Adds drive mode number *mode_id (0, 1, ... in call order = mode 1, 2, ... of Eq. 1) with
 * fundamental frequency omega (> 0) and Fourier truncation N_trunc (>= 0).  At most 4 modes. */
MMF_API int mmf_add_mode(mmf_sys* sys, double omega, int N_trunc, int* mode_id);
/* Sets V^{mode_id+1, harmonic} (D x D complex, any matrix; harmonic >= 1).  Harmonics of a
 * mode must be added in order 1, 2, ...; a missing harmonic is zero. */
MMF_API int mmf_add_coupling(mmf_sys* sys, int mode_id, int harmonic, const double* V);
MMF_API int mmf_sys_destroy(mmf_sys* sys);
/* Floquet dimension n = D prod (2 N_l + 1) (Sec. 2, Appendix A); -1 on a NULL handle. */
MMF_API int64_t mmf_dim(const mmf_sys* sys);
/* Half-bandwidth of H_F (Eq. 6, Appendix A): the largest |row - col| of a nonzero entry, from the
 * nonzero entries of H0 (|i - i'|) and of each harmonic h <= 2 N_l of mode l (D h S_l + i' - i,
 * S_l the block stride of mode l); at least 1; -1 on a NULL handle. */
MMF_API int mmf_sys_bandwidth(const mmf_sys* sys);

/* ---------------------------------------------------------------- one system (Sec. 3.2)
 * mmf_build: S1, assemble H_F on the device in the given precision (MMF_FP64 / MMF_MIXED);
 * *n_out = n.  Allocates the system's device state within the context budget. */
MMF_API int mmf_build(mmf_sys* sys, int precision, int64_t* n_out);
/* Copies the assembled H_F to the host: n x n complex, column-major (equal to row-major for
 * a Hermitian matrix up to conjugation: HF[c * n + r] = H_F(r, c)).  Must follow mmf_build
 * and precede mmf_diagonalise (the reduction overwrites it).  MIXED gives the FP32 matrix
 * widened to FP64. */
MMF_API int mmf_hamiltonian(mmf_sys* sys, double* HF);
/* S2-S6: full eigendecomposition of H_F on the device (the paper's LAPACK call, Sec. 3.2).
 * Returns the numerical status (MMF_ST_NOCONV if an iteration cap was hit). */
MMF_API int mmf_diagonalise(mmf_sys* sys);
/* All n quasienergies (eigenvalues of H_F), ascending, FP64. */
MMF_API int mmf_quasienergies(mmf_sys* sys, double* E);
/* Eigenvectors: n x n complex column-major, column k belongs to E[k]; entry (i + D b, k)
 * is <i, n_b | lambda_k>. */
MMF_API int mmf_eigenvectors(mmf_sys* sys, double* Z);
/* S7: U[k][j][i] = <j| U(t[k], t0) |i> for nt times (Eq. 3-5, summed over Floquet copies).
 * U is nt x D x D complex. */
MMF_API int mmf_time_evolution(mmf_sys* sys, double t0, int nt, const double* t, double* U);
/* S8: P[i * D + j] = Pbar_{i->j}, the average of |<j|U(t,t0)|i>|^2 over t and t - t0;
 * eigenvalues closer than 1e-8 max|E| are averaged as one degenerate cluster. */
MMF_API int mmf_transition_avg(mmf_sys* sys, double* P);
/* Micromotion operator of Eq. 5 for one Floquet zone: UF[k][j][a] = sum_n e^{-i n.w t_k}
 * <j, n | lambda_a> for the D eigenvectors with the largest weight on the central Fourier
 * block (ties to the lower eigenvalue), in ascending eigenvalue order; reps[a] receives
 * their eigenvalue indices (may be NULL). */
MMF_API int mmf_micromotion(mmf_sys* sys, int nt, const double* t, double* UF, int64_t* reps);
/* The paper's TIMEEVOLUTIONOPERATOR driver (Sec. 3.2): build + diagonalise + U in one call. */
MMF_API int mmf_time_evolution_operator(mmf_sys* sys, int precision, double t0, int nt,
                                const double* t, double* U);

/* ---------------------------------------------------------------- device-pointer variants
 * The same results as mmf_quasienergies, mmf_eigenvectors, mmf_time_evolution and
 * mmf_transition_avg (Sec. 3.2; Eq. 3-5 for U; the time average for Pbar), written into
 * caller-owned DEVICE memory (for example torch tensors) on the caller's CUDA stream `stream`
 * (a cudaStream_t; NULL = the legacy default stream) instead of host arrays.  Layouts as in the
 * host versions: E n doubles; Z n x n complex column-major (2 n^2 doubles); U nt x D x D complex
 * with U[k][j][i] = <j|U(t[k], t0)|i>; P D x D doubles, P[i * D + j] = Pbar_{i->j}.  For
 * mmf_time_evolution_dev the nt times t are device doubles, read in order after the work already
 * enqueued on `stream`.  The calls are asynchronous: the library's kernels run on the context's
 * stream, `stream` waits for them before the copy into the caller's buffer, and the context's
 * stream waits for that copy before any later library work.  The caller owns the buffers and
 * must keep them alive until `stream` has run the copy.  A change of nt re-plans the system
 * (its eigenpairs are recomputed, and that step waits on the host).  Errors: MMF_ERR_ARG (NULL
 * pointer, nt < 1), MMF_ERR_STATE (before mmf_diagonalise), MMF_ERR_CUDA. */
MMF_API int mmf_quasienergies_dev(mmf_sys* sys, double* E, void* stream);
MMF_API int mmf_eigenvectors_dev(mmf_sys* sys, double* Z, void* stream);
MMF_API int mmf_time_evolution_dev(mmf_sys* sys, double t0, int nt, const double* t, double* U, void* stream);
MMF_API int mmf_transition_avg_dev(mmf_sys* sys, double* P, void* stream);

/* ---------------------------------------------------------------- dressed basis (Sec. 3.3, Eq. 4)
 * Evolution expressed in the time-dependent basis of a subset of the modes (the "dressing" modes,
 * Sec. 3.3): with U_F(t) the micromotion operator of Eq. 5 for the system restricted to those
 * modes (one Floquet zone: its D eigenvectors of largest central-block weight, ties to the lower
 * index, in ascending order, as mmf_micromotion) and Ebar their quasienergies,
 *     Ud(t2, t1) = U_F(t2)^dagger U(t2, t1) U_F(t1),
 * where U(t2, t1) is the evolution of the full system (Eq. 3-4).  Without the other modes Ud is
 * diag(e^{-i Ebar (t2 - t1)}); with them it shows the transitions they drive between dressed
 * states (Sec. 4.1's probe spectroscopy).
 * mmf_sys_restrict: a new system (caller destroys it) with the same levels and H0 and only the
 *   modes listed in `modes` (indices in call order, each at most once), in that order.
 * mmf_batch_dressed: `full` is a batch of systems with nt >= 1 times t2 and start t0 = t1 (set by
 *   mmf_batch_set_times) and `dress` a batch, of the same count and levels, of the same systems
 *   restricted to their dressing modes (any nt); both have been run.  Writes (host, any may be
 *   NULL) Ud packed like the full batch's U (mmf_batch_dressed_offset(full, 0, i) in complex
 *   elements, nt x D x D per system, Ud[k][a][c] = <a|Ud(t2_k, t1)|c>) and Ebar (D doubles per
 *   system at mmf_batch_dressed_offset(full, 1, i)); mmf_batch_dressed_size(full, 0 or 1) gives
 *   the totals.  Waits for the result.  Errors: MMF_ERR_ARG (mismatched batches, nt = 0),
 *   MMF_ERR_STATE (a batch not run).
 * mmf_dressed_time_evolution: the same for one system: solves the restricted system and the
 *   full one (precision MMF_FP64 or MMF_MIXED) and writes Ud (nt x D x D complex) for the times
 *   t2[0..nt-1] from t1, and Ebar (D).  Returns the larger numerical status of the two solves. */
MMF_API int mmf_sys_restrict(const mmf_sys* sys, int nmodes, const int* modes, mmf_sys** out);
MMF_API int mmf_batch_dressed(mmf_batch* full, mmf_batch* dress, double* Ud, double* Ebar);
MMF_API int64_t mmf_batch_dressed_size(const mmf_batch* full, int what);
MMF_API int64_t mmf_batch_dressed_offset(const mmf_batch* full, int what, int i);
MMF_API int mmf_dressed_time_evolution(mmf_sys* sys, int ndress, const int* dressing, int precision, double t1,
                                       int nt, const double* t2, double* Ud, double* Ebar);

/* ---------------------------------------------------------------- spin systems (Sec. 3.4)
 * Coupling matrices of a spin S = S2/2 (D = S2 + 1 levels, basis m = S, S-1, ..., -S, angular
 * momentum matrices S_x, S_y, S_z as defined in Sakurai Sec. 3.5), built from the field
 * parameters of Eq. 7: three amplitudes A[i] and three phases phi[i] (i = x, y, z).
 *  - is_static = 0: the drive sum_i A_i cos(h w t + phi_i) S_i at one harmonic, written in
 *    mmf_add_coupling's convention (+ h.c. implied): V = sum_i (A_i / 2) e^{i phi_i} S_i.
 *    Eq. 7 prints the exponent without its i; it is read as a phase.  The cosine amplitude
 *    follows Eq. 8 and the example's field settings.
 *  - is_static = 1: the static part H0 = sum_i A_i S_i (phases ignored).
 * V: caller-owned, D x D row-major complex (2 D^2 doubles, interleaved re/im).  Host only, no
 * device or context needed.  Returns MMF_ERR_ARG for S2 < 1 or a NULL pointer. */
MMF_API int mmf_spin_components(int S2, const double* A, const double* phi, int is_static, double* V);

/* ---------------------------------------------------------------- batches
 * Many systems of any sizes solved together on the device (the data-parallel sweep of the
 * paper's examples, Sec. 4).  A batch is a plan: it allocates all device state once (within
 * the context budget) and can be run many times.  nt is the number of times per system.
 */
MMF_API int mmf_batch_create(mmf_ctx* ctx, int count, mmf_sys* const* systems, int precision, int nt,
                     mmf_batch** out);
/* Times: t is count x nt host doubles (row = system); t0 common to all. */
MMF_API int mmf_batch_set_times(mmf_batch* b, double t0, const double* t);
/* Re-uploads the systems' coefficients and the times from the host (pinned staging). */
MMF_API int mmf_batch_upload(mmf_batch* b);
/* Enqueues S1-S8 for every system on the context stream; returns without waiting. */
MMF_API int mmf_batch_run(mmf_batch* b);
/* enable != 0: the next mmf_batch_run captures the whole launch sequence (S1-S8) of the batch
 * into a CUDA graph, and later runs replay it with one graph launch.  Changing t0 or the timing
 * set-up re-captures.  enable = 0 returns to plain launches. */
MMF_API int mmf_batch_graph(mmf_batch* b, int enable);
/* Waits for the batch; status (count ints, may be NULL) receives each system's numerical
 * status.  Returns the largest status. */
MMF_API int mmf_batch_sync(mmf_batch* b, int* status);
/* Results of system i: E (n), U (nt x D x D complex), P (D x D); any may be NULL. */
MMF_API int mmf_batch_get(mmf_batch* b, int i, double* E, double* U, double* P);
/* Eigenvectors of system i (n x n complex column-major). */
MMF_API int mmf_batch_eigenvectors(mmf_batch* b, int i, double* Z);
/* Packed results of all systems (E: sum n, U: sum nt D^2 complex, P: sum D^2) copied to the
 * host with one transfer each; any may be NULL.  Enqueued and waited on the stream. */
MMF_API int mmf_batch_results(mmf_batch* b, double* E, double* U, double* P);
/* The packed results of mmf_batch_results copied into caller-owned DEVICE buffers on the
 * caller's stream (any may be NULL), ordered after the batch's work and before any later work
 * of the batch's stream; asynchronous (see the device-pointer variants above). */
MMF_API int mmf_batch_results_dev(mmf_batch* b, double* E, double* U, double* P, void* stream);
/* Offsets (in doubles for E and P, in complex elements for U) of system i in the packed
 * results: what = 0 (E), 1 (U), 2 (P). */
MMF_API int64_t mmf_batch_offset(const mmf_batch* b, int what, int i);
/* Total packed sizes: what = 0 (E doubles), 1 (U complex), 2 (P doubles). */
MMF_API int64_t mmf_batch_size(const mmf_batch* b, int what);
/* Per-stage CUDA-event timing: record events around the stages of the next max_runs calls
 * of mmf_batch_run (0 switches timing off).  mmf_batch_stage_ms waits for the stream and
 * returns in ms[MMF_STAGES] the summed times of the recorded runs per stage (0 assemble,
 * 1 small-n Jacobi, 2 Householder reduction, 3 tridiagonal eigensolve, 4 back-transform,
 * 5 refinement: H_F X, 6 refinement: FP64-accurate Gram products X^H X and X^H H_F X,
 * 7 refinement: the rest, 8 U and Pbar), *runs their number, and restarts the count. */
#define MMF_STAGES 9
MMF_API int mmf_batch_timing(mmf_batch* b, int max_runs);
MMF_API int mmf_batch_stage_ms(mmf_batch* b, double* ms, int* runs);
/* Eigensolver path of system i (returns one of MMF_PATH_*; *band, if not NULL, receives the
 * half-bandwidth used by the band path, else 0): the shared-memory Jacobi kernel, the dense
 * Householder reduction (one thread-block cluster per system), the whole-GPU dense reduction for
 * the largest systems, or the band path (bulge chase on the band of H_F, see MMF_OPT_BAND_MAX). */
#define MMF_PATH_JACOBI 0
#define MMF_PATH_DENSE 1
#define MMF_PATH_WHOLE_GPU 2
#define MMF_PATH_BAND 3
MMF_API int mmf_batch_path(const mmf_batch* b, int i, int* band);
/* Device bytes held by the batch. */
MMF_API size_t mmf_batch_bytes(const mmf_batch* b);
MMF_API int mmf_batch_destroy(mmf_batch* b);

/* ---------------------------------------------------------------- serving
 * Continuous batching of independent solve requests (the paper's parameter sweeps served as
 * they arrive).  A worker thread groups queued requests (same nt and the same size class of n as
 * the oldest waiting request: n <= 128, <= 640, <= 2500, larger; at most max_batch per plan) into
 * batch plans and runs each plan on one of `slots` CUDA streams; a plan is admitted only while
 * the context's HBM budget has room for it, so requests wait in the queue until slots and memory
 * free up.  Plans on different slots overlap on the device.  Finished plans stay resident (up to
 * max(4, 2 slots) of them, within the budget): a later group whose systems have the same
 * structure (levels, modes, truncations, harmonics, nt) reuses one, with its own coefficients and
 * times; resident plans are released, least recently used first, when a new plan needs memory.
 * Each request's results are those of the same system solved alone (up to summation order).
 *   mmf_serve_submit copies the system definition and the times; the caller may then change or
 *   destroy its system.  *ticket identifies the request.
 *   mmf_serve_wait blocks until the request is done (timeout_ms < 0: no limit; MMF_ERR_STATE on
 *   timeout), copies E (n), U (nt x D x D complex) and P (D x D) (any may be NULL), sets *status
 *   to the request's numerical status and releases the request.
 *   mmf_serve_stats: latency from submit to results-on-host of the requests completed since the
 *   last reset: median, 99th percentile and mean in ms, and their number.
 *   mmf_serve_destroy: finishes the plans in flight, drops queued requests; call it after every
 *   wait has returned. */
MMF_API int mmf_serve_create(mmf_ctx* ctx, int slots, int max_batch, int precision, mmf_server** out);
MMF_API int mmf_serve_submit(mmf_server* srv, const mmf_sys* sys, int nt, const double* t, double t0,
                             uint64_t* ticket);
MMF_API int mmf_serve_poll(mmf_server* srv, uint64_t ticket, int* done);
MMF_API int mmf_serve_wait(mmf_server* srv, uint64_t ticket, int timeout_ms, double* E, double* U,
                           double* P, int* status);
MMF_API int mmf_serve_stats(mmf_server* srv, double* p50_ms, double* p99_ms, double* mean_ms,
                            int64_t* completed);
MMF_API int mmf_serve_reset_stats(mmf_server* srv);
/* Plans created, plans reused from the resident set, and plans resident now (any may be NULL). */
MMF_API int mmf_serve_plan_stats(mmf_server* srv, int64_t* created, int64_t* reused, int64_t* resident);
MMF_API int mmf_serve_destroy(mmf_server* srv);

/* ---------------------------------------------------------------- no device allocation
 * No counterpart in the paper.  For callers that cannot allocate device memory (their HBM is
 * owned by another allocator, or they cannot afford cudaMalloc's implicit device
 * synchronisation): the eigenvalues and eigenvectors of one real symmetric tridiagonal matrix
 * tridiag(e, d, e), computed by the library's tridiagonal eigensolver (bisection + inverse
 * iteration, FP64) with all scratch taken from a fixed device array compiled into the library
 * (about 1.6 MB on every GPU that loads it, held until the process exits) instead of allocated.
 *   d  device, n doubles (diagonal);  e  device, n-1 doubles (off-diagonal; may be NULL if n == 1)
 *   E  device, n doubles: eigenvalues ascending;  Y  device, n*n doubles, row-major:
 *      Y[i*n + k] = component i of the eigenvector of E[k]
 *   status  device int or NULL: set to MMF_OK, or MMF_ST_NOCONV if a bisection reached its
 *      iteration cap (the caller reads it after the stream has run the call's work)
 *   stream: a cudaStream_t (NULL = the legacy default stream).
 * The call is asynchronous: it enqueues kernels on `stream` (no host copies, no allocation) and
 * returns.  n must be 1..MMF_NOALLOC_TRIDIAG_NMAX, otherwise MMF_ERR_UNSUPPORTED.  The first call
 * on a device (and the first after its context was reset) looks up the device address of the
 * scratch array, with that device current; make that first call before any stream capture.  All
 * calls share the scratch array: calls whose GPU work overlaps (other streams, other host
 * threads) race on it and must be serialised by the caller. */
#define MMF_NOALLOC_TRIDIAG_NMAX 256
MMF_API int mmf_tridiag_eig_noalloc(const double* d, const double* e, int n, double* E, double* Y,
                                    int* status, void* stream);

/* ---------------------------------------------------------------- diagnostics
 * Runs the library's batched tcgen05 GEMM (kind 0: TF32, kind 1: BF16; `products` copies of the
 * same product summed in one TMEM accumulator) on seeded M x K and N x K operands whose products
 * are exact, and compares C = products * A B^T with an FP64 reference computed on the device.
 * Returns the largest absolute difference and the largest |reference| entry.  Allocates its own
 * device memory; for health checks, not for the solve path. */
MMF_API int mmf_selftest_tensor_cores(int M, int N, int K, int kind, int products, double* max_abs_err,
                                      double* max_abs_ref);
/* Runs the mixed path's tensor-core Gram product G = X^H X (exact integer slicing of FP32 X on
 * the BF16 tensor cores) on one seeded n x n complex FP32 matrix (1 <= n <= 8192; entries over
 * six orders of magnitude) and compares it with an FP64 reference computed on the device.
 * Returns the largest absolute difference and the largest |reference| entry; allocates its own
 * device memory. */
MMF_API int mmf_selftest_gram(int n, double* max_abs_err, double* max_abs_ref);
/* Runs the split-TF32 tensor-core product used by the mixed path's refinement and back-transform
 * (each FP32 operand cut into two TF32 pieces, three products in one FP32 accumulator) on seeded
 * M x K and N x K FP32 operands with full 24-bit mantissas, in output mode 0 (store C = A B^T),
 * 1 (subtract A B^T from C) or 2 (write C's TF32 pieces as an operand; N a multiple of 32), and
 * compares with an FP64 reference computed on the device.  Returns the largest error relative to
 * sum_k |a_k b_k| of its entry, and the same for a sequential FP32 dot product (fmaf) for
 * comparison.  M x K, N x K and M x N at most 2^26 each; allocates its own device memory. */
MMF_API int mmf_selftest_split_tf32(int M, int N, int K, int mode, double* max_rel_err,
                                    double* max_rel_err_fp32);
/* Runs the mixed path's FP32 Householder reduction to tridiagonal form (Sec. 3.2's
 * diagonalisation, first step) on `count` seeded Hermitian n x n FP32 matrices in one launch
 * (2 <= n <= the one-CTA maximum, count <= 512, n^2 count <= 2^27), with the trailing update
 * A -= V W^H + W V^H on the tensor cores in split TF32 (tensor_cores = 1) or on the FP32 units
 * (0).  For the first two matrices the host applies the stored reflectors in FP64,
 * B = Q^H A Q, and returns max |B - tridiag(e, d, e)| over all entries and max |A|.  Allocates its
 * own device memory; for health checks, not for the solve path. */
MMF_API int mmf_selftest_hetrd(int n, int count, int tensor_cores, double* max_abs_err, double* max_abs_ref);

/* ---------------------------------------------------------------- misc */
MMF_API const char* mmf_strerror(int status);
MMF_API const char* mmf_last_error(void);
/* Number of kernel launches enqueued by the last mmf_batch_run on this thread. */
MMF_API int mmf_last_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* MMF_H */
