/*
 * lbm_gb300.h -- C ABI of the GB300 (sm_103a) coupled central-moment lattice Boltzmann
 * stepper for thermocapillary convection in superimposed fluid layers (arXiv 2210.07501).
 *
 * One time step advances three lattices at every node of an nx x ny channel:
 *   - the conservative Allen-Cahn phase field phi (Sec. 4.1; D2Q5 or D2Q9),
 *   - the two-fluid pressure/velocity lattice with the CSF surface-tension and Marangoni
 *     force (Sec. 4.2; D2Q9),
 *   - the energy lattice for T (Sec. 4.3; D2Q5 or D2Q9),
 * each collided in central-moment space through the maps P, F(u), F(-u), P^-1 of App. B
 * and streamed by a pull scheme, with sigma(T) = sigma0 + sigma1 (T - T_ref)
 * + sigma2 (T - T_ref)^2 (Sec. 2.3).
 *
 * Geometry (Sec. 2.1): periodic in x; walls at y = 0 (heated, T = T_hot + dT cos(2 pi k x /
 * nx)) and y = ny (T = T_cold), halfway between node rows; node (i, j) sits at x = i,
 * y = j + 1/2.  Flow walls are no-slip (bounce-back), the phase field has no flux through
 * the wall (specular reflection), temperature walls are Dirichlet (anti-bounce-back),
 * Sec. 5.1.  Fluid A (phi = 0) fills the bottom layer y < b, fluid B (phi = 1) the top.
 *
 * Conventions shared by every entry point:
 *   - Field arrays are row-major [ny][nx] doubles; row j = 0 is next to the heated wall,
 *     column i = 0 is under the heating peak.
 *   - Populations exchanged with the caller are [Q][ny][nx] doubles: f (phase field),
 *     g - w_a p0 (flow, p0 = rho_bottom / 3) and h - w_a T_ref (energy); "dp" is p - p0.
 *     Internally the phase field is stored as f - r_a(y), r the populations of the flat
 *     tanh interface of width W at y = b at rest (an exact change of variables that keeps
 *     round-off off the interface tilt); f is rebuilt as stored + r on output.
 *   - Every function returns LBM_OK (0) or a negative LBM_E* status and never throws.
 *     A handle is not thread-safe: use one handle per host thread.
 *   - The library owns all device memory it allocates; the caller owns every buffer it
 *     passes in.  Host pointers may be pageable or pinned.
 *   - Work is queued on the handle's CUDA stream; functions that return data to host
 *     memory synchronise that stream before returning.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define LBM_OK 0
#define LBM_EINVAL (-1)    /* bad argument, size or parameter                       */
#define LBM_ENOMEM (-2)    /* device or host allocation failed                       */
#define LBM_ECUDA (-3)     /* a CUDA call failed; lbm_strerror names it              */
#define LBM_EUNSTABLE (-4) /* a non-finite value appeared in the macroscopic fields  */
#define LBM_ETIMEOUT (-5)  /* run_to_steady reached max_steps before the tolerance   */
#define LBM_EIO (-6)       /* checkpoint file could not be read or written, or is bad */
#define LBM_EDEVICE (-7)   /* a step kernel gave up waiting (~1 s) for its own shared- */
                           /* memory copies; the state is invalid (never seen in use)  */

/* ---- storage precision of the populations (arithmetic: FP64 for LBM_FP64, else FP32) ---- */
#define LBM_FP64 0
#define LBM_FP32 1
#define LBM_FP16 2

/* ---- dtype of device field exports ---- */
#define LBM_DTYPE_F64 0
#define LBM_DTYPE_F32 1

typedef struct lbm_handle lbm_handle;

/* Lattice and discretisation (Sec. 2.1, Sec. 4). */
typedef struct {
    int32_t nx, ny;        /* nodes; nx >= 3, ny >= 3, ny * (nx rounded up to 64) < 2^31 */
    int32_t heat_periods;  /* cosine periods of the bottom-wall temperature along x (>= 0) */
    int32_t q_phi;         /* 5 or 9: phase-field lattice                                  */
    int32_t q_T;           /* 5 or 9: energy lattice                                       */
    int32_t precision;     /* LBM_FP64 | LBM_FP32 | LBM_FP16                                */
    double b;              /* height of the interface above the bottom wall (0 < b < ny)   */
    double W;              /* interface width (> 0)                                        */
} lbm_domain;

/* Fluid and thermal parameters (Sec. 2.2, 2.3, 3, 4). Lattice units. */
typedef struct {
    double sigma0, sigma1, sigma2;   /* sigma(T) = sigma0 + sigma1 (T-T_ref) + sigma2 (T-T_ref)^2 */
    double T_ref;                    /* reference temperature; also the initial T          */
    double T_hot, T_cold, dT;        /* bottom wall T_hot + dT cos(..), top wall T_cold     */
    double tau_flow;                 /* bottom fluid: nu = (tau_flow - 1/2) / 3  (> 1/2)    */
    double visc_ratio;               /* mu_top / mu_bottom (> 0)                            */
    double tau_T;                    /* bottom fluid: alpha = (tau_T - 1/2) / 3  (> 1/2)    */
    double cond_ratio;               /* k_top / k_bottom (> 0)                              */
    double tau_phi;                  /* mobility M_phi = (tau_phi - 1/2) / 3  (> 1/2)       */
    double rho_bottom, rho_top;      /* densities (> 0); c_p = 1                            */
    double Fx_ext, Fy_ext;           /* uniform external body force F_ext                   */
} lbm_params;

/* Create a solver, allocate its device state and initialise it at rest: tanh interface of
 * width W at y = b (Sec. 3), u = 0, T = T_ref, uniform pressure p0.  `stream` is a
 * cudaStream_t to queue work on (NULL: the library creates its own).  *out receives the
 * handle (NULL on failure).  Uses the current CUDA device. */
int lbm_create(const lbm_domain *domain, const lbm_params *params, void *stream, lbm_handle **out);

/* Re-initialise at the central-moment equilibrium of the given host fields [ny][nx]
 * (phi, u, v, T, dp = p - p0); a NULL field takes its default from lbm_create.  Resets
 * the step counter. */
int lbm_init_fields(lbm_handle *h, const double *phi, const double *u, const double *v,
                    const double *T, const double *dp);

/* Queue nsteps >= 0 time steps (Sec. 4.1-4.3: stream, moments, stencils, forces, collide).
 * Asynchronous; returns LBM_EINVAL / LBM_ECUDA only for launch-time errors.  Every
 * check_interval steps the macroscopic fields are stored and reduced (mass, residual). */
int lbm_step(lbm_handle *h, int64_t nsteps);

/* Macroscopic fields of the latest step (the values its collision used): phi = sum_a f_a
 * (Sec. 4.1), T = sum_a h_a (Sec. 4.3), the velocity rho c^2 u = sum_a g_a e_a + c^2 F_t / 2
 * and the pressure p = sum_a g_a + F_p . u / 2 (Sec. 4.2), returned as p - p0; into
 * caller-owned host arrays [ny][nx]; any pointer may be NULL.  Synchronises. */
int lbm_fields(lbm_handle *h, double *phi, double *u, double *v, double *T, double *dp);

/* As lbm_fields (the same macroscopic updates of Sec. 4.1-4.3), into caller-owned device
 * arrays [ny][nx] of LBM_DTYPE_F64 or LBM_DTYPE_F32 (e.g. torch tensors).  Asynchronous on
 * the handle's stream. */
int lbm_fields_device(lbm_handle *h, void *phi, void *u, void *v, void *T, void *dp, int dtype);

/* Global diagnostics (reductions with FP64 accumulation in a fixed order; the paper defines
 * no steady-state criterion, this residual is the library's own):
 * mass = sum of phi over the lattice at the current step; residual = ||u^n - u^{n-K}||_2 /
 * (K ||u^n||_2) over both components from the last two checks K steps apart (-1 before
 * two checks); step = steps taken.  Returns LBM_EUNSTABLE if a non-finite value was seen.
 * Synchronises. */
int lbm_diag(lbm_handle *h, double *mass, double *residual, int64_t *step);

/* Steps every check_interval (K >= 1) steps between residual checks; default 100 (no
 * counterpart in the paper). */
int lbm_set_check_interval(lbm_handle *h, int32_t K);

/* Step until residual <= tol or max_steps are taken; *steps_taken (may be NULL) receives
 * the count.  Returns LBM_OK, LBM_ETIMEOUT, LBM_EUNSTABLE or an error. Synchronises. */
int lbm_run_to_steady(lbm_handle *h, double tol, int64_t max_steps, int64_t *steps_taken);

/* Post-collision state (Sec. 4.1-4.3, after the collision of the latest step) in the
 * variables of the conventions above: f [q_phi][ny][nx], g [9][ny][nx], h [q_T][ny][nx],
 * dp [ny][nx] (pressure used by the next step's force).  g, h and dp round-trip exactly
 * through lbm_set_state / lbm_get_state in FP64 storage; f to within one rounding (it
 * passes through f - r). */
int lbm_get_state(lbm_handle *h, double *f, double *g, double *hT, double *dp);
int lbm_set_state(lbm_handle *h, const double *f, const double *g, const double *hT, const double *dp);

/* Checkpoint (no counterpart in the paper): the raw device state, step counter, domain,
 * parameters and a CRC32 of the payload.  lbm_load requires a file written for the same
 * domain (nx, ny, q_phi, q_T, precision, b, W) and tau_phi, which fix the phase-field
 * reference the state is stored against, and restores the state bit for bit.  LBM_EIO on
 * a missing, truncated, corrupt or mismatched file. */
int lbm_save(lbm_handle *h, const char *path);
int lbm_load(lbm_handle *h, const char *path);

/* Launch shape of the step kernel (no counterpart in the paper): each CTA walks `rows`
 * consecutive rows of a strip (0 = automatic: the length that minimises the waves of
 * resident CTAs times the rows each walks).  Affects speed only, never the results. */
int lbm_set_segment(lbm_handle *h, int32_t rows);

/* Test hook for the fault path (not part of the method).  The step kernel stages its
 * population rows in shared memory with asynchronous bulk copies and waits for them on
 * mbarriers with a limit of about one second; after the limit it flags a fault and
 * abandons the step instead of hanging.  With on != 0 every copy stage waits for 16 bytes
 * more than it copies, so the waits run out: the next lbm_step returns at once, the next
 * lbm_diag / lbm_fields (or batch step) returns LBM_EDEVICE after a few seconds, and the
 * state is invalid until lbm_init_fields, lbm_set_state or lbm_load.  on = 0 restores
 * normal stepping.  No GPU fault or trap is involved. */
int lbm_test_stall_copies(lbm_handle *h, int32_t on);

/* Autotuner (no counterpart in the paper): times `reps` launches of the step kernel for
 * each candidate segment length (the automatic choice, then 8 .. 256 rows below ny) and
 * keeps the fastest; *rows (may be NULL) receives its row count.  The kernel is re-launched
 * from the same input buffer, so the state and the step count are unchanged.
 * Synchronises. */
int lbm_autotune(lbm_handle *h, int32_t reps, int32_t *rows);

/* Bytes the step kernel moves per lattice node and step (populations read and written
 * once plus the stored pressure), for roofline accounting (no counterpart in the paper). */
int lbm_bytes_per_node(const lbm_handle *h, int64_t *bytes);

/* Number of step-kernel launches queued since creation (diagnostics; no counterpart in the
 * paper). */
int lbm_launch_count(const lbm_handle *h, int64_t *launches);

/* Largest node count lbm_reduce_fields_noalloc accepts. */
#define LBM_NOALLOC_MAX_NODES 2147483647LL

/* Field reductions for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a service of the library.  Who needs it: code that queues work
 * while its stream is being captured into a CUDA graph (cudaMalloc is not allowed there),
 * and plugins or custom calls inside a framework that owns every device allocation and
 * only hands over buffers.  The function allocates nothing: the caller passes the inputs
 * and the output, and the partial sums go to a 9.5 KiB scratch array compiled into the
 * library, which every GPU that loads the library keeps until the process exits.
 *
 * Inputs are caller-owned device arrays of n_nodes doubles (e.g. the fields written by
 * lbm_fields_device): phi, u, v, T, and optionally the velocity of an earlier step u_prev,
 * v_prev (both NULL: taken as zero).  result is a caller-owned device array of 4 doubles,
 * written on `stream` (a cudaStream_t; NULL = the legacy default stream):
 *   result[0] = sum phi, result[1] = sum (u - u_prev)^2 + (v - v_prev)^2,
 *   result[2] = sum u^2 + v^2, result[3] = number of nodes with a non-finite value,
 * summed in FP64 in the same fixed order as lbm_diag, so both give the same values.
 * Returns LBM_EINVAL for NULL inputs, for only one of u_prev / v_prev, or for n_nodes
 * outside 1 .. LBM_NOALLOC_MAX_NODES; LBM_ECUDA if a launch fails.  Asynchronous.
 *
 * The first call on each device looks up the scratch array's device address (with that
 * device current) and caches it; make that first call before any stream capture begins.
 * The cached address belongs to the device's context at that time: after
 * cudaDeviceReset (or anything else that destroys and recreates the primary context) it
 * is stale, so do not call this function again in such a process.
 * All calls on a device share the one scratch array: calls that overlap on the GPU (for
 * example on two streams at once) race and give wrong sums; serialise them.  Every call
 * overwrites all the scratch it reads, so leftovers of an earlier call do no harm. */
int lbm_reduce_fields_noalloc(const double *phi, const double *u, const double *v, const double *T,
                              const double *u_prev, const double *v_prev, int64_t n_nodes, double *result,
                              void *stream);

/* ---- batched parameter sweeps (many channels of uneven size, one launch per step) ---- */
typedef struct lbm_batch lbm_batch;

/* Create n independent channels (domains[c], params[c]; all with the same precision, q_phi
 * and q_T), each initialised as lbm_create does.  One step of the batch is one launch of
 * the step kernel over the strips of every still-active channel; chunks of K steps (one
 * residual check each) are captured once into a CUDA graph and replayed.  `stream` as in
 * lbm_create.  This is the batched sweep over (sigma1, sigma2, a/b, k~, mu~) of Sec. 6. */
int lbm_batch_create(int32_t n, const lbm_domain *domains, const lbm_params *params, void *stream, lbm_batch **out);

/* Steps per chunk and residual check (even, >= 2; default 100). */
int lbm_batch_set_check_interval(lbm_batch *b, int32_t K);

/* Autotuner for the batch launch: times `reps` launches per candidate segment length and
 * keeps the fastest (state untouched); *rows receives it.  Synchronises. */
int lbm_batch_autotune(lbm_batch *b, int32_t reps, int32_t *rows);

/* Advance every active channel by nsteps (a multiple of K).  Synchronises after every
 * chunk to read the per-channel residuals; LBM_EUNSTABLE if a channel went non-finite. */
int lbm_batch_step(lbm_batch *b, int64_t nsteps);

/* Step until every channel has residual <= tol (a converged channel stops being stepped)
 * or max_steps have been taken; steps[c] and converged[c] (arrays of n; may be NULL)
 * receive each channel's step count and status.  LBM_OK if all converged, else
 * LBM_ETIMEOUT (or an error). */
int lbm_batch_run_to_steady(lbm_batch *b, double tol, int64_t max_steps, int64_t *steps, int32_t *converged);

/* Fields, residual and step count of channel c (as lbm_fields); lbm_batch_init_fields
 * re-initialises channel c from host fields (as lbm_init_fields) and re-activates it. */
int lbm_batch_fields(lbm_batch *b, int32_t c, double *phi, double *u, double *v, double *T, double *dp);
int lbm_batch_diag(lbm_batch *b, int32_t c, double *residual, int64_t *steps);
int lbm_batch_init_fields(lbm_batch *b, int32_t c, const double *phi, const double *u, const double *v,
                          const double *T, const double *dp);
/* Number of channels, CTAs per batch launch and rows per CTA segment. */
int lbm_batch_size(const lbm_batch *b, int32_t *n, int32_t *ctas, int32_t *rows);
void lbm_batch_destroy(lbm_batch *b);

/* ---- learned warm start: a small convolutional surrogate of the steady fields ----
 * Not a step of the paper's method: it predicts the steady phi, u, v, T of a channel from
 * its parameters and heating profile, and its prediction initialises the LB solver
 * (lbm_init_fields), which then converges to the LB solution; the surrogate's error is
 * measured against that solution.
 * Network: six 3x3 convolutions, channels 12 -> 32 -> 32 -> 32 -> 32 -> 32 -> 4, SiLU between
 * layers, periodic in x, zero padding in y; FP32 weights, activations stored in BF16
 * (bf16_activations != 0) or FP32, FP32 accumulation.  Parameters, in order per layer:
 * weights [Cout][Cin][3][3], then biases [Cout].  Inputs x [B][12][H][W] and outputs /
 * targets [B][4][H][W] are caller-owned FP32 device arrays.  Deterministic. */
typedef struct lbm_cnn lbm_cnn;
int lbm_cnn_create(int32_t H, int32_t W, int32_t batch_max, int32_t bf16_activations, uint64_t seed, void *stream,
                   lbm_cnn **out);
int lbm_cnn_num_params(const lbm_cnn *c, int64_t *n);
int lbm_cnn_get_params(lbm_cnn *c, float *host);             /* host array of num_params floats */
int lbm_cnn_set_params(lbm_cnn *c, const float *host);       /* also resets the optimiser state */
int lbm_cnn_forward(lbm_cnn *c, const float *x, int32_t B, float *y);
/* Forward + backward of the mean squared error over all outputs: *loss (may be NULL) and
 * the gradient with respect to every parameter (grad_host, may be NULL).  Synchronises. */
int lbm_cnn_gradients(lbm_cnn *c, const float *x, const float *target, int32_t B, float *grad_host, double *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error. */
int lbm_cnn_train_step(lbm_cnn *c, const float *x, const float *target, int32_t B, float lr, double *loss);
const char *lbm_cnn_strerror(void);
void lbm_cnn_destroy(lbm_cnn *c);

/* Release the handle and its device memory; NULL-safe.  No counterpart in the paper
 * (resource management of the library). */
void lbm_destroy(lbm_handle *h);

/* Static string for a status code (for LBM_ECUDA, of the last CUDA error seen).  No
 * counterpart in the paper. */
const char *lbm_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
