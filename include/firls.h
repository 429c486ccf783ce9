/*
 * firls.h - C ABI of the GB300 (sm_103a) FIRLS library.
 *
 * FIRLS (fast iteratively reweighted least squares, arXiv 1411.5057) solves
 * the analysis-sparsity reconstruction problem (Eq. anapro / probogs / iso)
 *
 *     min_x  1/2 ||A x - b||^2 + lambda ||G Phi x||_{2,1}
 *                              + lambda_tv ||[D1 x, D2 x]||_{2,1}
 *
 * with A = R F an undersampled 2-D Fourier operator (R: sampling mask, F: the
 * unitary 2-D DFT), Phi an orthogonal periodic wavelet (Haar or
 * Daubechies-4, Mallat layout), G a group map built from rows of the
 * identity (Fig. 1) and D1/D2 first-order finite differences (Sec. 4.1, zero
 * extension at the image border).  Each outer step recomputes the weights
 * W (Eq. gw, Eq. Wog, Eq. wi) and runs preconditioned CG on the normal
 * equations (Eq. subprob, Eq. sub) with the pseudo-diagonal preconditioner
 * (Eq. pog) or, when TV is present, the penta-diagonal preconditioner with
 * the printed L U factors (Eq. ptv, Sec. 4.2) - Alg. 2 and Alg. 3.
 *
 * Conventions shared by every entry point:
 *   - Images are square, n x n, row-major; a batch is [batch][n][n].
 *   - Complex data is interleaved float pairs (re, im), i.e. complex64.
 *   - Every pointer documented as "device" must point to memory of the CUDA
 *     device that was current when the context was created; the caller
 *     keeps ownership of every buffer it passes in.
 *   - Work is enqueued on the context's stream; entry points return once
 *     the work is enqueued unless stated otherwise.
 *   - Errors are returned as firls_status codes, never thrown across the
 *     ABI.  Invalid arguments are rejected before any launch.  After an
 *     error the context stays valid; firls_last_error() gives a message.
 */
#ifndef FIRLS_H_
#define FIRLS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct firls_ctx firls_ctx;

typedef enum {
  FIRLS_OK = 0,
  FIRLS_E_INVALID_ARG = 1, /* null pointer, negative lambda, bad counts      */
  FIRLS_E_SHAPE = 2,       /* unsupported n, n not divisible by 2^levels ... */
  FIRLS_E_GROUPMAP = 3,    /* group index outside [0, n*n)                   */
  FIRLS_E_CUDA = 4,        /* a CUDA runtime call or kernel launch failed    */
  FIRLS_E_NOMEM = 5,       /* device allocation failed                       */
  FIRLS_E_BREAKDOWN = 6,   /* PCG breakdown (d^H S d <= 0 or not finite)     */
  FIRLS_E_STATE = 7,       /* call out of order (e.g. solve before operator) */
  FIRLS_E_DEVICE_TIMEOUT = 8 /* a bounded wait inside a kernel ran out; the
                                 slices it names hold invalid results        */
} firls_status;

/* Regulariser bitmask (psi_kind).  HAAR and DB4 are exclusive; TV
 * (isotropic, Eq. iso) or TV_ANISO (l1 TV, Eq. l1: ||D1 x||_1 + ||D2 x||_1,
 * weights W1 = (|D1 x|^2 + eps)^-1/2, W2 = (|D2 x|^2 + eps)^-1/2; Sec. 4.1
 * derives it like the isotropic form) may be combined with either wavelet, in
 * which case both terms enter S and the TV preconditioner's diagonal gains
 * lambda * diag(Phi^T W Phi).  TV and TV_ANISO are exclusive. */
enum { FIRLS_PSI_HAAR = 1, FIRLS_PSI_DB4 = 2, FIRLS_PSI_TV = 4, FIRLS_PSI_TV_ANISO = 8 };

/* Context flags. FIRLS_REAL_X: the unknown x is real (A^T y = Re F^H R^T y);
 * buffers are still complex64 and their imaginary parts are ignored on
 * input and written as 0 on output. */
enum { FIRLS_REAL_X = 1 };

/* Sizes accepted for n: 16, 32, 48, 64, 80, 96, 128, 160, 192, 256, 320,
 * 384, 512 (radix-2/3/5 FFT plans).  Query with firls_size_supported. */
int firls_size_supported(int n);

/* Create a context for `batch` independent slices of n_rows x n_cols
 * (square: n_rows == n_cols).  `cuda_stream` is a cudaStream_t (NULL = the
 * legacy default stream).  The context allocates its device workspace
 * (about 14 complex64 + 6 float vectors per slice) on the current device.
 * Returns FIRLS_E_SHAPE for unsupported sizes, FIRLS_E_NOMEM if the
 * workspace does not fit. */
firls_status firls_create(firls_ctx** out, int n_rows, int n_cols, int batch,
                          unsigned flags, void* cuda_stream);

/* Set the operator A and the regulariser (Alg. 2/3 inputs).
 *   mask        device uint8 [batch][n][n], 0/1, unshifted FFT order (DC at
 *               [0][0]); copied into the context.  mean(diag(A^H A)) of
 *               each slice is its popcount / n^2 (Sec. 5.4).
 *   psi_kind    FIRLS_PSI_* bitmask; a wavelet needs wavelet_levels >= 1
 *               with n divisible by 2^levels and n / 2^(levels-1) >= 2.
 *   group_idx   device int32: the Mallat-layout flat coefficient indices of
 *               the members of each group, group after group (the rows of
 *               G, Fig. 1; groups may overlap and may differ in size).
 *               NULL = singleton groups (plain l1: every coefficient is its
 *               own group, the IRLS weights of Sec. 3.1).
 *   group_off   device int32 [n_groups+1] CSR offsets into group_idx, or
 *               NULL for uniform groups of `group_size` members
 *               (group_idx is then [n_groups][group_size]).
 * The map is copied; the library builds the coefficient -> groups inverse
 * map (CSR, ascending group ids per coefficient) used to sum the
 * duplicated weights of Eq. Wog into diag(G^T W G) without atomics.
 * Synchronises the stream (reads back the popcounts and the map check).
 * Returns FIRLS_E_INVALID_ARG if a slice's mask is empty (popcount 0: A = 0,
 * nothing to reconstruct) and FIRLS_E_GROUPMAP if an index is outside
 * [0, n^2) or the offsets are not non-decreasing; after either error the
 * operator counts as not set. */
firls_status firls_set_operator(firls_ctx* ctx, const uint8_t* mask,
                                unsigned psi_kind, int wavelet_levels,
                                const int32_t* group_idx, const int32_t* group_off,
                                int n_groups, int group_size);

typedef struct {
  int outer_iters;  /* outer reweighting steps K (>= 1)                       */
  int pcg_iters;    /* PCG steps J per outer step (>= 1)                      */
  float pcg_tol;    /* stop PCG when ||r|| <= pcg_tol ||A^H b|| (0 = never)   */
  float outer_tol;  /* stop when ||x^{k+1}-x^k|| <= outer_tol ||x^k|| (0=never)*/
  float lambda;     /* wavelet lambda (lambda_W), >= 0                        */
  float lambda_tv;  /* TV lambda, >= 0 (ignored without FIRLS_PSI_TV)         */
  float eps;        /* smoothing eps of Eq. gw / Eq. wi; <= 0 selects 1e-10   */
  const float* lambda_per_slice;    /* host [batch] or NULL (use lambda)      */
  const float* lambda_tv_per_slice; /* host [batch] or NULL (use lambda_tv)   */
  int outer_tol_kind;  /* 0: stop when the relative change <= outer_tol;
                          1: stop when the estimated distance to the limit,
                          relchg * mu / (1 - mu) with the contraction
                          mu = (relchg_k / relchg_{k-24})^(1/24), at most
                          0.999 (linear convergence), and the relative change
                          are both <= outer_tol (after > 24 outer steps); with
                          a late inner schedule (pcg_iters_late > 0), also
                          once the relative change is <= outer_tol and has not
                          fallen by 20 % over the 24 outer steps before, all
                          taken from outer step outer_late on (the slice's
                          FP32 floor)                                         */
  int precond;         /* FIRLS_PRECOND_*: the PCG preconditioner (0 = the
                          paper's)                                            */
  float outer_stall_tol; /* stop a slice once its relative change has stayed
                          at or below this for 4 consecutive outer steps: the
                          FP32 rounding floor of the outer iteration, where
                          it cannot move closer (0 = never)                   */
  int pcg_tol_kind;    /* 0: pcg_tol is relative to ||A^H b||; 1: relative to
                          the first residual r_0 of each outer step (the
                          forcing term of an inexact inner solve: PCG runs
                          until ||r|| <= pcg_tol ||r_0|| or pcg_iters steps)  */
  int pcg_iters_late;  /* > 0: outer steps k >= outer_late (counted per slice
                          from 0) run this many PCG steps instead of
                          pcg_iters (a slice still running late has an
                          ill-conditioned subproblem whose outer rate needs a
                          nearly exact inner solve); 0 = pcg_iters throughout */
  int outer_late;
  int boundary_period; /* outer-step transitions and weight updates run in
                          every this-many-th macro step (0 or 1: every one);
                          a slice waits at most boundary_period - 1 macro
                          steps per outer step, and the mostly idle set-up
                          launches run that much less often                  */
} firls_params;

/* Preconditioners of the PCG steps, for the comparison of Sec. 5.2 (Fig. 2
 * and the TV figure).  PAPER: the proposed P (Eq. pog: Phi^T (abar I +
 * lambda G^T W G)^{-1} Phi without TV; Eq. ptv with the printed L U factors of
 * Sec. 4.2 with TV).  JACOBI: P = diag(S) = abar + lambda diag(Phi^T G^T W G
 * Phi) + lambda_tv diag(D1^T W D1 + D2^T W D2).  NONE: P = I (standard CG).
 * ILU0 (TV only): the penta-diagonal P of Eq. ptv factored by the incomplete
 * LU with zero fill and updated pivots, d_i = a_i - P_{i,i-1}^2 / d_{i-1}
 * - P_{i,i-n}^2 / d_{i-n}, L = I + L_P diag(d)^{-1}, U = diag(d) + U_P (L U
 * equals P on P's pattern; the printed factors keep d = a). */
enum { FIRLS_PRECOND_PAPER = 0, FIRLS_PRECOND_JACOBI = 1, FIRLS_PRECOND_NONE = 2, FIRLS_PRECOND_ILU0 = 3 };

typedef struct {
  int outer_done;            /* outer steps run (max over slices)             */
  long long pcg_steps;       /* PCG steps run, summed over slices             */
  double max_rel_change;     /* max_s ||x^{K}-x^{K-1}|| / ||x^{K-1}||         */
  double max_rel_residual;   /* max_s ||r|| / ||A^H b|| at the last PCG step  */
  int n_breakdown;           /* slices stopped by a PCG breakdown             */
} firls_stats;

/* How the solver advances (every entry point below that iterates): each slice
 * moves through its own outer steps independently.  One "macro step" (a
 * fixed launch sequence, captured as a CUDA graph) gives every slice one step
 * of its outer step: the start of an outer step (weights W^k and P from x^k,
 * S x^k, the first residual r_0, z_0 = P^{-1} r_0) or one PCG step (S d,
 * alpha, x/r update, z = P^{-1} r, beta), or, for a slice whose PCG has
 * stopped, the end of the outer step (x^{k+1} = x^k + sum_j alpha_j d_j, the
 * relative change, the stopping rules) followed by the start of its next
 * one.  A slice's PCG stops after pcg_iters steps or at its tolerance, so
 * slices with different inner step counts never wait for each other.  An
 * outer step with J PCG steps spans J + 1 macro steps. */

/* Run FIRLS on every slice (Alg. 2 / Alg. 3).
 *   b      device complex64 [batch][n][n] k-space, entries off the mask are
 *          ignored (multiplied by the mask).
 *   x0     device complex64 [batch][n][n] warm start, or NULL for
 *          x^1 = A^H b (Sec. 3.3).
 *   x_out  device complex64 [batch][n][n]; receives x^{K+1}.
 *   stats  host, may be NULL.  When non-NULL, or when a tolerance is set,
 *          the call synchronises the stream before returning.
 * Operators run in FP32; the PCG inner products, alpha, beta, rho, the
 * residual norms and the relative change are accumulated in FP64.
 * Returns FIRLS_E_BREAKDOWN if any slice broke down (its x_out holds its
 * last iterate; the other slices are unaffected).  A slice whose A^H b is
 * not finite (a NaN or infinity in b on the mask) is not iterated and counts
 * as a breakdown; its x_out holds its start (x0, or A^H b).  b = 0 is not a
 * breakdown: x = 0 is then exact and PCG stops at rho = 0. */
firls_status firls_solve(firls_ctx* ctx, const void* b, const firls_params* params,
                         const void* x0, void* x_out, firls_stats* stats);

/* Solve several contexts (slices of different sizes, e.g. 128^2 .. 320^2)
 * together: one outer step of every context is captured as ONE CUDA graph
 * (forked from ctxs[0]'s stream onto each context's own stream and joined
 * back) and replayed outer_iters times on ctxs[0]'s stream.  Arrays have
 * n_ctx entries, params included (per-context lambdas); the schedule,
 * tolerances and boundary_period must be equal in all of them (with
 * boundary_period P > 1 the captured outer step holds a boundary stage every
 * P-th macro step, as in firls_solve).  Contexts must have distinct,
 * non-default streams for the graph; otherwise the steps are enqueued
 * directly.  Same buffer rules as firls_solve; results are ordered on
 * ctxs[0]'s stream.  stats (host, may be NULL) has n_ctx entries. */
firls_status firls_solve_multi(firls_ctx* const* ctxs, int n_ctx,
                               const void* const* b, const firls_params* params,
                               const void* const* x0, void* const* x_out,
                               firls_stats* stats);

/* Message for the last error on this context (static storage owned by the
 * context; valid until the next call on it). */
const char* firls_last_error(const firls_ctx* ctx);

/* Free the context and its device workspace (synchronises its stream). */
void firls_destroy(firls_ctx* ctx);

/* ---- operator-level entry points (for tests and roofline measurement) ----
 * All act on device buffers of the context's batch and run on its stream. */

/* q = A^H A d (unitary FFT, mask, inverse FFT; Sec. 5.4 A = RF). */
firls_status firls_apply_AHA(firls_ctx* ctx, const void* d, void* q);

/* c = Phi x (Mallat layout; wavelet of the context). */
firls_status firls_apply_Phi(firls_ctx* ctx, const void* x, void* c);

/* x = Phi^T c. */
firls_status firls_apply_PhiT(firls_ctx* ctx, const void* c, void* x);

/* Update the weights from x (Eq. gw + Eq. Wog, Eq. wi) and the
 * preconditioner (Eq. pog / Eq. ptv); then q = S d and z = P^{-1} r.
 * lambda/lambda_tv/eps are taken from params (per-slice arrays allowed). */
firls_status firls_apply_S_P(firls_ctx* ctx, const firls_params* params,
                             const void* x, const void* d, void* q,
                             const void* r, void* z);

/* ---- continuous batching (serving) ----
 * Slots of a context hold independent slices at different stages of their
 * solve.  A slice that has converged (outer_tol) or reached the caller's cap
 * is read out and its slot reloaded with the next slice while the other
 * slots keep iterating, so throughput follows the average number of outer
 * steps per slice instead of the slowest slice of a fixed batch.
 *
 * firls_slot_load: put one slice into slot s: copy its mask (device uint8
 *   [n][n]) and k-space b (device complex64 [n][n]), compute its A^H b and
 *   popcount, start from x0 (device, one slice) or A^H b, reset its state
 *   with its own lambdas (eps <= 0 selects 1e-10).  Other slots untouched.
 *   Reads back the popcount (synchronises the stream): an empty mask returns
 *   FIRLS_E_INVALID_ARG and leaves the slot retired.
 * firls_run: enqueue sum_k (J_k + 1) + 1 macro steps (J_k the PCG steps of
 *   outer step k, k < params->outer_iters) for every slot that is not done:
 *   a slot that starts its first outer step at the first of them completes
 *   params->outer_iters outer steps; no host synchronisation.
 * firls_run_steps: enqueue `macro_steps` macro steps (one captured graph,
 *   cached per schedule and count); no host synchronisation.
 * firls_slot_status: per-slot done flag, outer steps, last relative change
 *   and PCG steps (host arrays [batch], each may be NULL); synchronises.
 * firls_slot_retire: slot s stops taking part until reloaded.
 * firls_slot_get: copy slot s's current x (device complex64 [n][n]). */
firls_status firls_slot_load(firls_ctx* ctx, int s, const uint8_t* mask, const void* b, const void* x0,
                             float lambda, float lambda_tv, float eps);
firls_status firls_run(firls_ctx* ctx, const firls_params* params);
firls_status firls_run_steps(firls_ctx* ctx, const firls_params* params, int macro_steps);
firls_status firls_slot_status(firls_ctx* ctx, int* done, int* outer_done, double* rel_change, int* pcg_steps);
firls_status firls_slot_retire(firls_ctx* ctx, int s);
firls_status firls_slot_get(firls_ctx* ctx, int s, void* x_out);

/* Slot compaction for the end of a queue, when few slots still run and most
 * launched blocks would find their slot idle (no counterpart in the paper).
 * firls_slot_move: slot `from` continues in slot `to` (every per-slice array
 *   and its state are copied on the stream; `from` is retired).  `to` must
 *   not hold a running slice (it is overwritten).  Results are bit for bit
 *   those of the unmoved slice.
 * firls_set_active_slots: firls_run_steps and firls_run launch only slots
 *   [0, k) (k = 0 or batch: all); slots >= k must not hold a running slice
 *   (they are left as they are).  The other entry points always cover the
 *   whole batch.  FIRLS_E_INVALID_ARG for k outside [0, batch]. */
firls_status firls_slot_move(firls_ctx* ctx, int from, int to);
firls_status firls_set_active_slots(firls_ctx* ctx, int k);

/* Autotuner: time the tile-shape choices of this context's size, batch and
 * regulariser on its own buffers (CUDA events on its stream) and keep the
 * fastest: the wavelet form (1, 2: every level of a slice in one launch on a
 * thread-block cluster, the weights staged in shared memory or read from
 * HBM, where the slice fits; 4, 8, 16: rows per CTA of the tiled levels), the
 * largest wavelet block kept in shared memory by the tiled form (32, 64), the
 * ILU shared-memory ring
 * shape (10 * rows per stage + stages: 42, 43, 44, 22, 23, 24, as far as
 * they fit).  cache_path (may be NULL) is a text file of earlier
 * results keyed by "n batch psi levels": a hit skips the timing, a miss
 * appends the new result.  Overwrites the context's workspace; call after
 * firls_set_operator and before solving.  Synchronises the stream. */
firls_status firls_autotune(firls_ctx* ctx, const char* cache_path);

/* Multi-contrast images (Sec. 5.6, FIRLS_MT and FIRLS_JTV): with channels
 * C > 1, every C consecutive slices of the batch are the contrasts x_1..x_C
 * of one cross section, each with its own mask (set_operator) and k-space.
 * They share the regulariser's weights: joint wavelet sparsity, W_j =
 * (sum_t |(Phi x_t)_j|^2 + eps)^(-1/2) (non-overlapping groups across the
 * contrasts, Eq. gw), and joint TV, W_i = (sum_t |grad_1 x_t,i|^2 +
 * |grad_2 x_t,i|^2 + eps)^(-1/2).  Given W the system and P are block
 * diagonal over the contrasts, and PCG runs on the stacked unknown: the inner
 * products, the PCG stop, the relative change and the outer stop are sums
 * over an image's contrasts, so its C slices move in lockstep (same outer
 * and PCG counts).  firls_objective returns each image's F_eps for every one
 * of its slices.  The contrasts of an image must share lambda and lambda_tv
 * (FIRLS_E_INVALID_ARG from the solve otherwise).  Not with a group map or
 * FIRLS_PSI_TV_ANISO, and not with the slot API (FIRLS_E_STATE from
 * firls_slot_load).  channels must divide the batch; 1 (the default) is the
 * single-contrast solver.  Call before solving; no device work. */
firls_status firls_set_channels(firls_ctx* ctx, int channels);

/* Failure-detection test hook (no counterpart in the paper).  With enable = 1
 * the TV preconditioner kernel (the ILU sweeps of Sec. 4.2) of every later
 * outer step runs in a test form: its producer issues no copy and every
 * bounded wait between its warps gives up after the first poll.  The waits
 * run out with nothing in flight, the slices are marked faulted and
 * firls_solve returns FIRLS_E_DEVICE_TIMEOUT; the context stays usable.
 * enable = 0 restores the normal kernel.  Only contexts with FIRLS_PSI_TV
 * launch that kernel. */
firls_status firls_set_wait_test(firls_ctx* ctx, int enable);

/* The tile shapes in use (0 = built-in default). */
firls_status firls_get_tuning(const firls_ctx* ctx, int* rows_per_cta, int* coarse_max, int* ilu_depth);

/* Set the tile shapes explicitly (0 = built-in default for that shape):
 * the wavelet form (1 or 2: the one-launch cluster form as above; 4, 8 or
 * 16: rows per CTA of the tiled levels; the default is the cluster form with
 * staged weights where a slice fits, else 8 rows), the largest wavelet block
 * kept in shared memory by the tiled form, and the ILU ring shape (10 * rows
 * per stage + stages).  FIRLS_E_INVALID_ARG if a shape does not exist or does
 * not fit this size.  A captured outer
 * step is re-captured at the next solve. */
firls_status firls_set_tuning(firls_ctx* ctx, int rows_per_cta, int coarse_max, int ilu_shape);

/* atb = A^H b = F^H R^T b (real unknown: its real part), the zero-filled
 * reconstruction and x^1 of Sec. 3.3.  b, atb device complex64 [batch][n][n]. */
firls_status firls_adjoint(firls_ctx* ctx, const void* b, void* atb);

/* out = F^H((1 - R) F x + R b): keeps x's unsampled k-space and restores the
 * measured entries (data consistency of a warm start; A out = b exactly, so
 * its data term of F is zero like that of A^H b).  b, x, out device complex64
 * [batch][n][n]; out may alias x.  Real unknown: the real part. */
firls_status firls_data_consistency(firls_ctx* ctx, const void* b, const void* x, void* out);

/* F_eps(x) per slice: 1/2 ||A x - b||^2 + lambda sum_g sqrt(||(G Phi x)_g||^2 + eps)
 * + lambda_tv sum_i sqrt(|(D1 x)_i|^2 + |(D2 x)_i|^2 + eps) (Eq. anapro / iso with the
 * eps of Eq. gw / wi; Theorem 2 says FIRLS never increases it).  b, x device
 * complex64 [batch][n][n]; out host double [batch]; lambdas / eps from params.
 * Synchronises the stream. */
firls_status firls_objective(firls_ctx* ctx, const void* b, const firls_params* params, const void* x,
                             double* out);

/* Warm-start guard of the learned variant: per slice, x0 = x1 when
 * F_eps(x1) <= F_eps(A^H b), otherwise x0 = A^H b (the plain start).  x1, x0
 * device complex64 [batch][n][n] (x0 may not alias x1); chosen (host int
 * [batch], may be NULL) receives 1 where x1 was kept.  Synchronises. */
firls_status firls_warm_start_guard(firls_ctx* ctx, const void* b, const firls_params* params, const void* x1,
                                    void* x0, int* chosen);

/* Copy out the current per-coefficient wavelet weights diag(G^T W G)
 * (device float [batch][n][n]), the TV weights W (W1 for l1 TV) and, for l1
 * TV only, W2 (device float [batch][n][n] each); any pointer may be NULL
 * (w_tv2 must be NULL without FIRLS_PSI_TV_ANISO: FIRLS_E_STATE). */
firls_status firls_get_weights(firls_ctx* ctx, float* w_wavelet, float* w_tv, float* w_tv2);

/* Copy out the TV preconditioner's diagonal pieces of the last outer step
 * (Eq. ptv with the wavelet term of the combined TV + wavelet case):
 * wavelet_diag = diag(Phi^T W Phi) (needs a wavelet term) and inv_a = 1/a,
 * a = abar + lam_tv (D1^T W D1 + D2^T W D2)_ii + lam diag(Phi^T W Phi)_i.
 * Device float [batch][n][n] each; either may be NULL.  FIRLS_E_STATE
 * without FIRLS_PSI_TV. */
firls_status firls_get_precond(firls_ctx* ctx, float* wavelet_diag, float* inv_a);

/* Copy out the inverse group map (device int32: offsets [n*n+1], ids
 * [total members]).  FIRLS_E_STATE if no group map is set. */
firls_status firls_get_inverse_map(firls_ctx* ctx, int32_t* offsets, int32_t* ids);

/* Per-slice mask popcounts M (device int32 [batch]). */
firls_status firls_get_popcounts(firls_ctx* ctx, int32_t* counts);

/* ---- per-kernel timing (instrumentation for roofline measurement) ----
 * Kernel classes of one outer step. */
enum {
  FIRLS_K_ROW_FFT = 0,       /* d = z + beta d, row FFT                       */
  FIRLS_K_COL_FFT_MASK = 1,  /* column FFT, mask, column IFFT                 */
  FIRLS_K_WAVELET_S = 2,     /* Phi^T (w o Phi d), the wavelet term of S      */
  FIRLS_K_WAVELET_P = 3,     /* Phi^T (pinv o Phi r), the wavelet P^{-1}      */
  FIRLS_K_ROW_IFFT = 4,      /* row IFFT + TV stencil + wavelet term + dot    */
  FIRLS_K_ILU = 5,           /* x, r update and the two triangular sweeps     */
  FIRLS_K_AXPY = 6,          /* x, r update                                   */
  FIRLS_K_SCALARS = 7,       /* FP64 alpha / beta / rho / outer bookkeeping   */
  FIRLS_K_WEIGHTS = 8,       /* weights, group sums, diag(Phi^T W Phi), P set-up */
  FIRLS_K_OTHER = 9,         /* copies, relative change                       */
  FIRLS_NKCLASS = 10
};

/* Enable (1) or disable (0) CUDA-event timing of every kernel launch of the
 * macro steps on the context's stream (the events are recorded into the
 * captured macro-step graph).  Adds one event pair per launch group. */
firls_status firls_set_timing(firls_ctx* ctx, int enable);

/* Per-class totals over the macro steps of the last graph captured with
 * timing on and then executed (for firls_solve: one outer step, J + 1 macro
 * steps): ms[FIRLS_NKCLASS] milliseconds, launches[FIRLS_NKCLASS] kernel
 * launches and applications[FIRLS_NKCLASS] launch groups (one operator
 * application each; may be NULL).  Synchronises the stream.  FIRLS_E_STATE if
 * timing is off or nothing ran. */
firls_status firls_get_timing(firls_ctx* ctx, double* ms, int* launches, int* applications);

/* ---- learned warm start (not in the paper; workload of the learned variant) ----
 * A 6-layer 3x3 CNN (3 -> 32 -> 32 -> 32 -> 32 -> 32 -> 2 channels, ReLU between
 * layers, zero padding) maps [Re A^H b, Im A^H b, mask] to a correction:
 * x1 = A^H b + CNN(.), used as the FIRLS warm start (firls_solve's x0).  BF16
 * weights and activations (NHWC), FP32 accumulation on the tensor cores, FP32
 * master weights with Adam (beta 0.9 / 0.999, eps 1e-8).  Loss: sum |x1 - x*|^2. */
typedef struct firls_cnn firls_cnn;

/* Network for `batch` images of n x n (n a multiple of 32); allocates
 * weights, optimiser state and activations on the current device.  The
 * parameters are undefined until firls_cnn_set_params. */
firls_status firls_cnn_create(firls_cnn** out, int n, int batch, void* cuda_stream);

/* Set the FP32 parameters (host arrays, one per layer): w[l] is
 * [3][3][c_in][c_out] (row tap, column tap, input, output channel), b[l]
 * [c_out].  Resets the Adam state.  Synchronises the stream. */
firls_status firls_cnn_set_params(firls_cnn* net, const float* const* w, const float* const* b);

/* Copy the FP32 parameters / the last step's gradients to host arrays
 * (same layout; NULL entries are skipped).  Synchronise the stream. */
firls_status firls_cnn_get_params(firls_cnn* net, float* const* w, float* const* b);
firls_status firls_cnn_get_grads(firls_cnn* net, float* const* dw, float* const* db);

/* x1 = A^H b + CNN([Re A^H b, Im A^H b, mask]) for the batch: atb and x1
 * device complex64 [batch][n][n], mask device uint8 [batch][n][n]. */
firls_status firls_cnn_forward(firls_cnn* net, const void* atb, const uint8_t* mask, void* x1);

/* One training step on the batch: forward (x1 written), loss
 * sum |x1 - target|^2, backward, Adam update with learning rate lr.
 * target device complex64 [batch][n][n]; loss (host, may be NULL) receives
 * the loss before the update (synchronises when non-NULL). */
firls_status firls_cnn_train_step(firls_cnn* net, const void* atb, const uint8_t* mask, const void* target,
                                  void* x1, float lr, double* loss);

void firls_cnn_destroy(firls_cnn* net);

/* ---- allocation-free A^H A (no counterpart in the paper) ----
 * For callers that must not allocate device memory (code running inside
 * another framework's memory pool or a real-time loop, where cudaMalloc /
 * cudaFree would synchronise the device or break a fixed memory budget, and
 * plug-ins that are handed only their input and output buffers).
 *
 * q = A^H A d for `batch` slices of n x n (same operation and kernels as
 * firls_apply_AHA, without a context): mask device uint8 [batch][n][n],
 * d and q device complex64 [batch][n][n], caller-owned; runs on the given
 * stream (NULL = legacy default stream).
 *
 * Scratch: instead of allocating, the library keeps fixed-size __device__
 * arrays (FFT intermediate of FIRLS_NOALLOC_MAX_ELEMS complex values, a
 * twiddle table, per-slice state and partial sums: 8.4 MiB) that every
 * GPU loading the library holds until the process exits.  Limits:
 * batch * n * n <= FIRLS_NOALLOC_MAX_ELEMS and batch <= FIRLS_NOALLOC_MAX_BATCH;
 * larger requests return FIRLS_E_SHAPE, as do unsupported n.  Null pointers
 * return FIRLS_E_INVALID_ARG; a failed CUDA call FIRLS_E_CUDA.
 *
 * The first call on a device (it looks up the arrays' device addresses),
 * and every call whose n differs from the previous call's on that device
 * (it rewrites the twiddle table from a host buffer and synchronises the
 * stream), must be made outside stream capture.  All calls share the same
 * arrays, which keep the last call's contents; each call rewrites what it
 * reads before reading it.  Calls that overlap on the GPU (different
 * streams, or different host threads) race on the arrays: serialise them.
 * The host-side set-up is guarded by a lock, so first calls from several
 * host threads are safe.  A CUDA error makes the next call redo the set-up;
 * a cudaDeviceReset in the process is not supported (the cached addresses
 * and the twiddle table are not refreshed after it).
 * No cudaMalloc, cudaFree or allocating library routine is called. */
#define FIRLS_NOALLOC_MAX_ELEMS (1 << 20)
#define FIRLS_NOALLOC_MAX_BATCH 64
firls_status firls_apply_AHA_noalloc(int n, int batch, const uint8_t* mask, const void* d, void* q,
                                     void* cuda_stream);

/* ---- Dense sensing matrix (Sec. 5.2-5.3: random projections) -----------
 *
 * FIRLS_L1 with a dense real A in place of the partial Fourier operator:
 *     min_x 1/2 ||A x - b||^2 + lambda ||x||_1,  A in R^{M x N}, x in R^N
 * (Eq. anapro with Phi = I and singleton groups).  Alg. 2 with W =
 * diag((x_i^2 + eps)^(-1/2)) (Eq. gw), S = A^T A + lambda W (Eq. subprob) and
 * the proposed preconditioner P = abar I + lambda W, abar = tr(A^T A) / N, the
 * mean diagonal entry of A^T A (Eq. ps, Eq. pog with Phi = I); Jacobi PCG
 * uses P = diag(A^T A) + lambda W and plain CG P = I (Sec. 5.2).
 *
 * A context holds `problems` independent problems of one shape.  With
 * shared_matrix = 0 every problem has its own A (A device float
 * [problems][M][N]); with 1 all problems share one A ([M][N]) and differ in b
 * (several signals measured by one projection).  Vectors are device float:
 * b [problems][M], x [problems][N].  Constraints: 1 <= M, 4 <= N <= 8192 with
 * N % 4 == 0 (rows are read as 16-byte vectors; A 16-byte aligned),
 * 1 <= problems <= 65535 with problems * M and problems * N below 2^31
 * (FIRLS_E_SHAPE otherwise).  Operators run in FP32; the PCG
 * inner products, alpha, beta, rho, the residual norms and the relative change
 * in FP64.  With a matrix per problem each step S d = A^T (A d) + lambda W d
 * streams A once (a row's product with d is formed and immediately scattered
 * back along the row); with a shared matrix and M % 4 == 0, A^T A d for all
 * problems is two register-tiled GEMMs, T = D A^T and Q = T A. */
typedef struct firls_dense_ctx firls_dense_ctx;

firls_status firls_dense_create(firls_dense_ctx** out, int M, int N, int problems, int shared_matrix,
                                void* cuda_stream);
/* Copy A (device float, see above; the context keeps its own copy) and
 * compute diag(A^T A) and abar per matrix.  Synchronises the stream. */
firls_status firls_dense_set_matrix(firls_dense_ctx* ctx, const float* A);
/* abar per matrix (host double [shared_matrix ? 1 : problems]).  Synchronises. */
firls_status firls_dense_abar(firls_dense_ctx* ctx, double* out);
/* q = A^T A d per problem (device float [problems][N] each; q may not alias
 * d).  The operator-level entry point of the parity tests and the bandwidth
 * measurement. */
firls_status firls_dense_apply_AtA(firls_dense_ctx* ctx, const float* d, float* q);
/* Run FIRLS_L1 on every problem from x^1 = A^T b (x0 NULL) or x0.  Uses
 * params->outer_iters, pcg_iters, pcg_tol (relative to ||A^T b||),
 * outer_tol (relative change), lambda / lambda_per_slice, eps and precond
 * (PAPER, JACOBI or NONE); every other field must be 0 (FIRLS_E_INVALID_ARG).
 * Problems advance independently (each stops on its own tolerance).  Returns
 * FIRLS_E_BREAKDOWN if a problem broke down (x_out holds its last iterate);
 * a problem whose A^T b is not finite is not iterated and counts as one.
 * stats (host, may be NULL) as for firls_solve.  Synchronises the stream. */
firls_status firls_dense_solve(firls_dense_ctx* ctx, const float* b, const firls_params* params, const float* x0,
                               float* x_out, firls_stats* stats);
const char* firls_dense_last_error(const firls_dense_ctx* ctx);
firls_status firls_dense_destroy(firls_dense_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* FIRLS_H_ */
