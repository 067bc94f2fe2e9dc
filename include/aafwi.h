/*
 * aafwi.h -- C ABI of the GB300 (sm_103a) library for the hot path of
 * Anderson-accelerated seismic inversion (Yang, "Anderson Acceleration for
 * Seismic Inversion", 2020): the adjoint-state FWI / LSRTM gradient of the
 * 2D constant-density acoustic wave equation and the l2 Anderson step on the
 * steepest-descent fixed-point map.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Every call returns an int status: AAFWI_OK (0) or one of AAFWI_ERR_*.
 *    No C++ exception crosses this boundary.  aafwi_last_error() returns a
 *    human-readable message for the last failure on a plan (or, for a NULL
 *    plan, the last failure of a create call on this thread).
 *  * Arrays named "device" are CUDA device pointers owned by the caller, of
 *    FP32 unless stated.  Arrays named "host" are ordinary host pointers.
 *  * Model-sized arrays are the PHYSICAL grid, row-major [nz][nx] (x fastest).
 *  * Trace arrays are CSR by shot: shot s occupies trace_count_s = nt_s*nrec_s
 *    consecutive floats starting at the sum of the counts of shots 0..s-1,
 *    time-major [nt_s][nrec_s].  Sample n of a trace is u^{n+1} (n = 0..nt_s-1).
 *  * `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on it, except that a non-NULL `*_host` output makes the
 *    call synchronise the stream before returning.
 *  * All arithmetic runs in this library's CUDA kernels; there is no CPU
 *    fallback.  Workspace (wavefield history or checkpoints, per-shot image
 *    accumulators, traces, reduction partials) belongs to the plan and is
 *    allocated once by aafwi_plan_create with cudaMalloc (the staging
 *    buffers of aafwi_adjoint_gradient_host on its first call).
 *  * A plan is used by one host thread at a time, and its calls run in the
 *    order they are made on one stream: the workspace is shared by all of
 *    them.  Internally a per-step sweep may fork onto the plan's own lane
 *    streams and joins back to the caller's stream before the call returns
 *    its work to it.
 *
 * Discretisation (the paper leaves it open; this library's reading):
 *   u^{n+1} = G (2 u^n - G u^{n-1} + W (L u^n + s^n)),  u^0 = u^{-1} = 0,
 *   W = dt^2 / m on the padded grid (model edge-replicated into an nb-cell
 *   sponge on all four sides), G = g(d_z) g(d_x) with g(d) = exp(-(0.015 d)^2)
 *   for a cell d cells into the sponge, L the 8th-order 5-point-per-axis
 *   Laplacian with zero values outside the padded grid, s^n the Ricker sample
 *   w(t_n) / (dx dz) at the source cell.
 */
#ifndef AAFWI_H
#define AAFWI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define AAFWI_OK            0
#define AAFWI_ERR_ARG       1   /* invalid argument (NULL, size, index, duplicate) */
#define AAFWI_ERR_CFL       2   /* c_max*dt/min(dx,dz) above the stability limit 0.55 */
#define AAFWI_ERR_OOB       3   /* source / receiver outside the physical grid */
#define AAFWI_ERR_NAN       4   /* model has a non-finite or non-positive value */
#define AAFWI_ERR_TIMEOUT   5   /* a bounded device-side wait ran out.  A persistent sweep's
                                   neighbour wait: the call fails, the plan stays usable.  A
                                   per-step kernel's tile-copy (TMA) wait or a U-Net tensor-core
                                   wait: a copy or an MMA may still have been in flight when the
                                   CTA returned, so the plan / network is retired -- every later
                                   call on it returns AAFWI_ERR_TIMEOUT; destroy it and reset the
                                   device context (cudaDeviceReset) before going on */
#define AAFWI_ERR_CUDA      6   /* a CUDA runtime call failed */
#define AAFWI_ERR_NOMEM     7   /* workspace does not fit the budget / device */
#define AAFWI_ERR_STATE     8   /* call out of order (e.g. reuse without a stored forward) */

/* adjoint_gradient modes */
#define AAFWI_MODE_FWI      0   /* unknown m = 1/c^2:  J = 1/2||F(m) - d||^2  (eq. FWI) */
#define AAFWI_MODE_LSRTM    1   /* unknown rho, m_r = rho m0: J = 1/2||L rho - d||^2 (eq. LSRTM) */

/* adjoint_gradient flags */
#define AAFWI_REUSE_FORWARD 1   /* skip the forward pass: the last aafwi_model_forward
                                   on this plan (FWI) ran on the same model contents */

typedef struct aafwi_plan aafwi_plan;
typedef struct aafwi_aa aafwi_aa;
typedef void *aafwi_stream;     /* cudaStream_t */

/* Grid: nx, nz physical cells; nb sponge cells on each side; spacing (m);
 * time step (s); c_max = largest velocity the plan will see (m/s), used for
 * the CFL check at creation. */
typedef struct {
    int nx, nz, nb;
    double dx, dz, dt;
    double c_max;
} aafwi_grid;

/* Shots (host arrays, copied at creation): S shots; source cell (physical
 * iz, ix); record length nt[s] (steps); receivers in CSR form rec_off[S+1]
 * into rec_iz/rec_ix (physical cells).  Receivers of one shot must be
 * distinct cells. */
typedef struct {
    int S;
    const int *src_iz, *src_ix;
    const int *nt;
    const int *rec_off;
    const int *rec_iz, *rec_ix;
} aafwi_shots;

/* Plan options (all zero = defaults). */
typedef struct {
    size_t max_workspace_bytes;  /* 0: 85% of the free device memory at creation */
    int checkpoint_every;        /* 0: planner picks (1 = keep every step if it fits,
                                    else k ~ sqrt(2 nt)); 1: force full history */
    int tile_z, tile_x;          /* 0: defaults / autotuned; else a supported tile */
    int engine;                  /* AAFWI_ENGINE_*: how FWI sweeps are launched */
    int no_graphs;               /* 0: the per-step sweeps (one launch per time step) are
                                    captured into CUDA graphs once per plan, sweep kind and
                                    caller buffer, and replayed; 1: launched kernel by kernel */
    int shots_per_batch;         /* 0: planner picks -- all shots if their workspace fits, else
                                    batches of shots run one after another (full history while a
                                    batch still fills the GPU, else checkpoints); > 0: this many */
    int no_pdl;                  /* 0: each per-step launch after the first of a sweep is a
                                    programmatic dependent launch (it becomes resident while the
                                    previous step drains; same results); 1: plain launches */
    int steps_per_launch;        /* FWI forward sweeps with the full history on the per-step
                                    engine: 0 or 1 = one time step per launch; 2 = two (the tile
                                    and a 4-cell ring advanced to n+1 on chip, then the tile to
                                    n+2; bitwise the one-step results, fewer launches and L2
                                    reads but 1.6x the stencil work of the first step: slower
                                    on the workloads measured).  Born sweeps and checkpoint
                                    plans always take one. */
    int lanes;                   /* per-step sweeps: the batch's shots in this many groups (0 = 4,
                                    at most 8; fewer if the batch has fewer shots) whose launch
                                    chains run on forked streams, so that one group's step
                                    boundary (grid drain, dependency wait, refill) overlaps the
                                    others' work; same results for any value */
    int l2_batches;              /* shot batches sized for the L2: the most shots whose adjoint
                                    working set (z^{n+1}, z^{n+2}, image) fits 40% of the L2,
                                    split evenly.  0: only when the plan runs batches anyway
                                    (memory); 1: always -- for workloads that reuse no stored
                                    forward, such as LSRTM gradients (a one-batch FWI plan
                                    would lose AAFWI_REUSE_FORWARD); -1: never.  Ignored when
                                    shots_per_batch is set; same results for any value */
} aafwi_plan_opts;

/* plan engines */
#define AAFWI_ENGINE_AUTO       0   /* per step (the fastest on the workloads measured;
                                       aafwi_autotune chooses per geometry) */
#define AAFWI_ENGINE_PER_STEP   1   /* one launch per time step (all shots) */
#define AAFWI_ENGINE_PERSISTENT 2   /* one cooperative launch per sweep; ARG if the
                                       plan does not qualify (full history, strips of
                                       the shots' rows fitting shared memory) */
#define AAFWI_ENGINE_HYBRID     3   /* forward sweeps per step, adjoint sweeps as one
                                       cooperative launch (same conditions) */

typedef struct {
    int NZ, NX, pitch;           /* padded grid and row pitch (floats) */
    int S, nt_max;
    long long trace_count;       /* total floats of a CSR trace array */
    int checkpoint_every;        /* 1 = full history kept */
    int n_checkpoints;
    size_t workspace_bytes;
    int tile_z, tile_x;
    int n_tiles;                 /* tiles per shot */
    int engine;                  /* AAFWI_ENGINE_PER_STEP, _PERSISTENT or _HYBRID */
    int persist_ctas;            /* strips of the persistent sweeps (0 if per step) */
    int shots_per_batch, n_batches;   /* the plan's shot batches (1 batch: all shots at once;
                                         more: the stored forward is not kept between calls,
                                         AAFWI_REUSE_FORWARD returns STATE) */
    int steps_per_launch;        /* time steps per launch of the per-step FWI forward sweeps */
    int lanes;                   /* shot lanes of the per-step sweeps */
} aafwi_plan_info;

/* ---- plan -------------------------------------------------------------- */

/* Build a plan on the current CUDA device (Sec. 2.2 problem statement:
 * geometry of eq. FWD and the sampling operator R of eq. FWI).
 * wavelet: host FP64 [max nt], the source time function w(t_n), n = 0..max nt-1.
 * Errors: ARG (NULL/size/duplicate receivers), OOB, CFL, NOMEM, CUDA. */
int aafwi_plan_create(const aafwi_grid *grid, const aafwi_shots *shots,
                      const double *wavelet, const aafwi_plan_opts *opts,
                      aafwi_plan **out);
void aafwi_plan_destroy(aafwi_plan *plan);
int aafwi_plan_get_info(const aafwi_plan *plan, aafwi_plan_info *info);
const char *aafwi_last_error(const aafwi_plan *plan);

/* Failure-detection test hook (not part of the method): from sweep step
 * `step` on, strip 0 of the persistent sweeps stops publishing its progress,
 * so its neighbours' bounded waits run out (about a second) and the call
 * reports AAFWI_ERR_TIMEOUT; the CUDA context stays usable.  step < 0 turns
 * the hook off.  STATE if the plan has no persistent sweeps. */
int aafwi_plan_set_stall(aafwi_plan *plan, int step);

/* ---- wave-equation operators (Sec. 2.2) -------------------------------- */

/* F: m -> R F(m) (eqs. FWD, FWI).  m: device [nz][nx] (s^2/m^2); d_out:
 * device CSR traces or NULL.  Stores the forward wavefield history (or its
 * checkpoints) in the plan so that a following adjoint_gradient with
 * AAFWI_REUSE_FORWARD can skip its forward pass. */
int aafwi_model_forward(aafwi_plan *plan, const float *m, float *d_out, aafwi_stream stream);

/* L: rho -> scattered traces (eq. Born, perturbation m_r = rho * m0).
 * m0, rho: device [nz][nx]; d_out: device CSR traces. */
int aafwi_born_forward(aafwi_plan *plan, const float *m0, const float *rho,
                       float *d_out, aafwi_stream stream);

/* Residual and misfit (eq. FWI): resid = d_syn - d_obs (device CSR, may be
 * NULL), J = 1/2 sum resid^2 accumulated in FP64.  J_host NULL: J stays on the
 * device (aafwi_read_misfit). */
int aafwi_misfit(aafwi_plan *plan, const float *d_syn, const float *d_obs,
                 float *resid, double *J_host, aafwi_stream stream);

/* Adjoint-state gradient (eqs. FWI_adj, adj_grad1).
 * FWI:   m = model (device [nz][nx]), rho NULL; grad = dJ/dm.
 * LSRTM: m = background m0, rho = current reflectivity; grad = L^T(L rho - d_obs).
 * d_obs: device CSR traces; grad: device [nz][nx]; J_host as in aafwi_misfit.
 * flags: AAFWI_REUSE_FORWARD (FWI only). */
int aafwi_adjoint_gradient(aafwi_plan *plan, int mode, const float *m, const float *rho,
                           const float *d_obs, float *grad, double *J_host, int flags,
                           aafwi_stream stream);

/* The same gradient with host buffers: the whole round trip in one call.
 * m, rho: host [nz][nx] (rho NULL for FWI); d_obs: host CSR traces; grad:
 * host [nz][nx] (out); J_host required.  The call copies m, rho and d_obs
 * into plan-owned device staging buffers (allocated on first use), runs
 * aafwi_adjoint_gradient on them, copies grad back and returns after the
 * stream has synchronised.  Pinned host memory makes the copies DMA on the
 * stream; pageable memory also works.  The stored forward belongs to the
 * staging buffer, so AAFWI_REUSE_FORWARD is not offered here.
 * Errors: as aafwi_adjoint_gradient; NOMEM if the staging buffers cannot be
 * allocated. */
int aafwi_adjoint_gradient_host(aafwi_plan *plan, int mode, const float *m, const float *rho,
                                const float *d_obs, float *grad, double *J_host, aafwi_stream stream);

/* Adjoint-state gradient for an arbitrary adjoint source (the data-space
 * derivative dJ/df of any misfit, Sec. 2.2 eq. FWI_adj): grad = (dF/dm)^T adj_src.
 * m: device [nz][nx]; adj_src: device CSR traces; grad: device [nz][nx].
 * flags: AAFWI_REUSE_FORWARD as in aafwi_adjoint_gradient. */
int aafwi_fwi_adjoint(aafwi_plan *plan, const float *m, const float *adj_src, float *grad,
                      int flags, aafwi_stream stream);

/* L^T: residual traces -> image on the physical grid (RTM image when
 * resid = d_r; Sec. 4.3 start model m_RTM = L^T d_r). */
int aafwi_born_adjoint(aafwi_plan *plan, const float *m0, const float *resid,
                       float *img, aafwi_stream stream);

/* Copy the last misfit J (FP64) computed on this plan to the host (syncs). */
int aafwi_read_misfit(aafwi_plan *plan, double *J_host, aafwi_stream stream);

/* ---- Anderson acceleration (Sec. 2.1, Sec. 3, Alg. 2) ------------------ */

/* State for AA(M) on n unknowns with the fixed step eta of eq. GD: a ring of
 * the last M+1 accepted iterates p_i and gradients G_i (FP32, device) and
 * their FP64 Gram matrix.  Allocates on the current device. */
int aafwi_aa_create(size_t n, int M, double eta, aafwi_aa **out);
void aafwi_aa_destroy(aafwi_aa *aa);
int aafwi_aa_set_eta(aafwi_aa *aa, double eta);

/* Damping beta in [0, 1] of the AA point (Alg. 1 eq. AAupdate0): p_tilde =
 * (1 - beta) sum alpha_i p_i + beta sum alpha_i G(p_i), i.e. the gamma form
 * with eta scaled by beta; p_bar keeps eta.  Default 1 (Alg. 2).  ARG if
 * beta is outside [0, 1]. */
int aafwi_aa_set_beta(aafwi_aa *aa, double beta);

/* Norm of the optimisation step (Sec. 2.1: eq. AAopt may use the l1, l2 or
 * l-infinity norm; the first and the last need linear programming).
 * AAFWI_NORM_L2 (default) is the least squares of Alg. 2 step 2.  With
 * AAFWI_NORM_L1 / AAFWI_NORM_LINF, aa_step takes the columns the l2 rank
 * safeguard keeps and solves gamma = argmin || W (dG gamma - G_k) ||_1 or _inf
 * (W the diagonal of aa_set_weights, identity without): the n rows stay on
 * the GPU, each round is one pass over the ring, and the host solves a linear
 * programme in the Mk+1 unknowns -- l-infinity by an exact working-set method
 * (rows above the current level are added until none is left), l1 by cutting
 * planes on sum |r_i| until the best value and the lower bound agree to a
 * relative gap of 1e-9.  Both are bounded by a box of 1e3 x max(1, |gamma_l2|)
 * around zero; a solution on that box returns AAFWI_ERR_STATE.  These steps
 * synchronise the stream.  May be changed between steps.  Errors: ARG, NOMEM
 * (first switch to l1 / l-infinity allocates the round buffers). */
#define AAFWI_NORM_L2   0
#define AAFWI_NORM_L1   1
#define AAFWI_NORM_LINF 2
int aafwi_aa_set_norm(aafwi_aa *aa, int norm);

/* Statistics of the last l1 / l-infinity step: the optimal value found
 * (sum or max of |W (dG gamma - G_k)|), the LP lower bound, rounds (passes
 * over the ring) and LP rows (cuts for l1, working-set rows for l-infinity). */
typedef struct {
    double objective;
    double lower_bound;
    int rounds;
    int rows;
} aafwi_aa_lp_info;
int aafwi_aa_get_lp_info(const aafwi_aa *aa, aafwi_aa_lp_info *info);

/* The host LP solver of the l1 / l-infinity steps, exposed for testing:
 * x = argmin c^T x subject to A x <= b, x free; A row-major [m][nv]
 * (1 <= nv <= 64), b [m], c [nv]; x [nv] and *obj (may be NULL) receive the
 * optimum.  Revised simplex on the dual with Bland's rule.  Host memory
 * only; no device call.  Errors: ARG, STATE (unbounded, infeasible or an
 * iteration limit; aafwi_last_error(NULL) says which). */
int aafwi_lp_min(int nv, int m, const double *A, const double *b, const double *c, double *x, double *obj);

/* Weighted l2 norm for the AA least-squares problem (Sec. 2.1): gamma =
 * argmin sum_i w_i ((dG gamma - G_k)_i)^2 with the device FP32 weights w [n]
 * (w_i >= 0; copied, the caller keeps its buffer); NULL restores the plain l2
 * norm.  Only before the first aa_step (the Gram matrix is built
 * incrementally with these weights): STATE otherwise. */
int aafwi_aa_set_weights(aafwi_aa *aa, const float *w, aafwi_stream stream);

/* Alg. 2 steps 1-3: append (p_k, grad_k) to the history (dropping the
 * oldest beyond M+1), then
 *   p_bar   = p_k - eta grad_k                                   (eq. GD)
 *   gamma   = argmin || [G_{i+1} - G_i]_i gamma - G_k ||_2        (eqs. Ak, solveGamma)
 *   p_tilde = p_bar - sum_i gamma_i [(p_{i+1} - eta G_{i+1}) - (p_i - eta G_i)]
 *                                                                (eq. AA2_update)
 * gamma is solved in FP64 from the Gram matrix of the history gradients
 * (Cholesky; while min R_jj < 1e-6 max R_jj the oldest column is dropped).
 * p_k, grad_k: device [n] (read); p_tilde, p_bar: device [n] (written).
 * gamma_host (len >= M) / Mk_host: optional host outputs (sync when given). */
int aafwi_aa_step(aafwi_aa *aa, const float *p_k, const float *grad_k, float *p_tilde,
                  float *p_bar, double *gamma_host, int *Mk_host, aafwi_stream stream);

/* Alg. 2 step 5: p_next = clip(lambda p_tilde + (1 - lambda) p_bar, lo, hi)
 * (no clip when lo >= hi).  armijo_dot_host (optional, syncs) receives
 * <G_k, p_next - p_k> in FP64 for the sufficient-decrease test of step 4. */
int aafwi_aa_combine(aafwi_aa *aa, double lambda, const float *p_tilde, const float *p_bar,
                     float *p_next, float lo, float hi, double *armijo_dot_host,
                     aafwi_stream stream);

/* max_i |x_i| of a device FP32 vector (FP64 result on the host, syncs);
 * used to fix eta = factor * max|p_0| / max|grad J(p_0)|.  Its scratch (and
 * aafwi_dot's) is one small library-owned buffer per device, allocated by the
 * first call on that device and reused; calls from several host threads are
 * serialised.  Errors: ARG (NULL, n = 0), NOMEM (first call), CUDA. */
int aafwi_absmax(const float *x, size_t n, double *host_out, aafwi_stream stream);

/* ---- learned preconditioner (not part of the paper) ---------------------- */

/* A U-Net (4 levels, base width C; 3x3 convolutions with ReLU, 2x2 max
 * pooling, 2x2 stride-2 transposed convolutions, skip concatenation, 1x1
 * head) mapping a 2-channel image [normalised gradient, normalised model] to
 * a 1-channel model update.  BF16 weights and NHWC activations on tensor
 * cores with FP32 accumulation, FP32 master weights, Adam.
 * Parameter vector layout (FP32, host): for each of the 17 convolutions in
 * network order (enc0a, enc0b, enc1a, enc1b, enc2a, enc2b, bottom a, bottom b,
 * then per decoder level 2, 1, 0: upconv, dec a, dec b) the weights then the
 * bias; 3x3 weights [Cout][3][3][Cin], upconv weights [Cin][2][2][Cout];
 * then the head weights [C] and bias [1]. */
typedef struct aafwi_unet aafwi_unet;

/* Allocate a network for batches up to Bmax of H x W images (H, W multiples
 * of 8) with base width C (multiple of 8).  Parameters start at zero: set them
 * with aafwi_unet_set_params. */
int aafwi_unet_create(int Bmax, int H, int W, int C, aafwi_unet **out);
void aafwi_unet_destroy(aafwi_unet *net);
long long aafwi_unet_param_count(const aafwi_unet *net);
/* Copy n FP32 parameters from / to the host (n = param_count); set resets Adam. */
int aafwi_unet_set_params(aafwi_unet *net, const float *host, long long n);
int aafwi_unet_get_params(aafwi_unet *net, float *host, long long n);
/* y[B][H][W] = net(x[B][2][H][W]); device FP32 arrays. */
int aafwi_unet_forward(aafwi_unet *net, const float *x, int B, float *y, aafwi_stream stream);
/* Loss 1/(2 B H W) sum (net(x) - target)^2 and its parameter gradient
 * (device FP32 [param_count], may be NULL); loss_host optional (syncs). */
int aafwi_unet_loss_grad(aafwi_unet *net, const float *x, const float *target, int B, float *grad,
                         double *loss_host, aafwi_stream stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on that loss with learning rate lr. */
int aafwi_unet_train_step(aafwi_unet *net, const float *x, const float *target, int B, float lr,
                          double *loss_host, aafwi_stream stream);

/* One 3x3 convolution GEMM of the network (cross-correlation, zero padding
 * 1) on BF16 operands with FP32 accumulation, as the forward and backward
 * passes run it; device arrays, NHWC activations, raw BF16 bits.
 *   AAFWI_CONV3_FWD   a = x [B][H][W][Cin], b = w [Cout][3][3][Cin]
 *                     -> out [s][B H W][Cout]  (y = conv(x, w), no bias)
 *   AAFWI_CONV3_DGRAD a = dz [B][H][W][Cout], b = wt [Cin][3][3][Cout] (w with
 *                     its channel axes swapped) -> out [s][B H W][Cin] (dL/dx)
 *   AAFWI_CONV3_WGRAD a = dz [B][H][W][Cout], b = x [B][H][W][Cin]
 *                     -> out [s][Cout][3][3][Cin]  (dL/dw)
 * The result is the sum of the s slices (split K); s is written to
 * *splits_used (may be NULL).  splits: at most this many slices (<= 0: the
 * network's own choice); out_cap: floats available at out, at least one
 * result (the slices used never exceed it).  Synchronises the stream.
 * Errors: AAFWI_ERR_ARG for bad sizes, AAFWI_ERR_TIMEOUT when a tensor-core
 * wait ran out (the device context must then be reset). */
#define AAFWI_CONV3_FWD 0
#define AAFWI_CONV3_DGRAD 1
#define AAFWI_CONV3_WGRAD 2
int aafwi_unet_conv3x3(int op, const void *a, const void *b, int B, int H, int W, int Cin, int Cout, int splits,
                       float *out, long long out_cap, int *splits_used, aafwi_stream stream);

/* Network input of the learned step from a gradient and a model (device FP32
 * [nz][nx]): stats (device double[3]) = (max|grad|, mean m, std m) and
 * x[2][H][W] = (grad / max|grad|, (m - mean) / std) on the top-left nz x nx
 * corner of the H x W network grid, zero elsewhere. */
int aafwi_learned_features(const float *grad, const float *m, int nz, int nx, int H, int W, float *x,
                           double *stats, aafwi_stream stream);
/* Learned step: out = clip(m + std_m * delta[:nz, :nx], lo, hi) (no clip when
 * lo >= hi); delta is the network output [H][W], stats from
 * aafwi_learned_features. */
int aafwi_learned_apply(const float *m, const float *delta, int nz, int nx, int W, const double *stats, float lo,
                        float hi, float *out, aafwi_stream stream);

/* ---- misfit without device allocation ----------------------------------- */

/* The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they run -- a host framework that owns
 * the whole device budget through its own pool or caching allocator, or a
 * latency-bound loop that must not pay the device-wide synchronisation of
 * cudaMalloc / cudaFree.
 *
 * Same result as aafwi_misfit (resid = d_syn - d_obs, J = 1/2 sum resid^2 in
 * FP64; partial sums over fixed chunks, so the last bits of J may differ from
 * aafwi_misfit's), without a plan and without allocating: the scratch (FP64
 * partial sums and J) is a 512 KB file-scope __device__ array of the library,
 * held on every GPU that loads the library until the process exits.
 *   d_syn, d_obs: device FP32 [n]; resid: device FP32 [n] or NULL;
 *   J_dev: device double (written on the stream) or NULL; J_host: host double
 *   (the call synchronises the stream) or NULL; at least one of the two.
 * n must lie in [1, AAFWI_MISFIT_NOALLOC_MAX_SAMPLES]; larger inputs return
 * AAFWI_ERR_ARG with a message (aafwi_last_error(NULL)) and launch nothing.
 * Every call looks up the array's address on the current device
 * (cudaGetSymbolAddress, a host-side query); the first call on a device may
 * also load the library's kernels there, so make that first call before any
 * stream capture.  All calls share the one array and every call overwrites it, so
 * calls whose kernels overlap on the GPU (other streams, other host threads)
 * race: serialise them on one stream. */
#define AAFWI_MISFIT_NOALLOC_MAX_SAMPLES (1LL << 32)
int aafwi_misfit_noalloc(const float *d_syn, const float *d_obs, long long n, float *resid,
                         double *J_dev, double *J_host, aafwi_stream stream);

/* ---- instrumentation ---------------------------------------------------- */

/* ---- vector operations of the comparison solvers (Sec. 5: restarted GMRES on
 * the LSRTM normal equations, L-BFGS for FWI) ------------------------------ */

/* <x, y> of two device FP32 vectors of length n, accumulated in FP64 in a
 * fixed order (deterministic); result on the host (syncs the stream).  Uses
 * the per-device reduction scratch of aafwi_absmax (no allocation after the
 * first call on a device).  Errors: ARG (NULL, n = 0), NOMEM, CUDA. */
int aafwi_dot(const float *x, const float *y, size_t n, double *host_out, aafwi_stream stream);

/* y = a x + b y on device FP32 vectors of length n (a, b rounded to FP32);
 * asynchronous on the stream.  x and y may be the same vector.
 * Errors: ARG, CUDA (launch). */
int aafwi_axpby(double a, const float *x, double b, float *y, size_t n, aafwi_stream stream);

/* y = clip(a x + b y) to [lo, hi] (no clip when lo >= hi): the bound
 * constraint applied to a trial point of a line search.  Asynchronous.
 * Errors: ARG, CUDA (launch). */
int aafwi_axpby_clip(double a, const float *x, double b, float *y, size_t n, float lo, float hi,
                     aafwi_stream stream);

/* ---- autotuner (launch configuration of the sweeps; the paper has no
 * counterpart) ------------------------------------------------------------ */

typedef struct {
    int engine;      /* AAFWI_ENGINE_PER_STEP, _PERSISTENT or _HYBRID */
    int tile_z;      /* tile rows of the per-step forward (16, 32 or 64); 0 for PERSISTENT */
    int lanes;       /* shot lanes of the per-step sweeps (aafwi_plan_info.lanes of the plan) */
    double ms;       /* median CUDA-event time of one forward sweep plus one FWI
                        adjoint sweep reusing it, over the first `steps` steps */
} aafwi_tune_entry;

/* Time the launch configurations a plan of this geometry may use and return
 * the fastest as plan options.  Candidates: the per-step engine with each tile
 * height, and, when a plan with these options keeps the full history and its
 * strips fit on chip, the persistent engine and the hybrid engine with each
 * tile height (base->engine, when not AUTO, restricts the candidates to that
 * engine); all with the default shot lanes, then, unless base->lanes fixes
 * them, the winner with 1, 2 and 8 lanes.  Each candidate is a temporary
 * plan over the same shots (over the first batch of shots when a plan of the
 * full record would run them in batches) with every record length cut to `steps` (the
 * sweeps' time grows in proportion to the steps), timed `reps` times after one
 * warm-up on the device model m [nz][nx] (FP32, m = 1/c^2) with zero observed
 * data, on a stream of its own.
 * base: options copied into *best (NULL = defaults), which gets the winner's
 * engine and tile_z; table: the first table_cap candidates timed (may be NULL
 * when table_cap is 0); *n_entries: number of candidates timed.
 * Synchronises the device.  Errors: ARG, CFL, NAN (model), NOMEM, CUDA. */
int aafwi_autotune(const aafwi_grid *grid, const aafwi_shots *shots, const double *wavelet,
                   const float *m, int steps, int reps, const aafwi_plan_opts *base,
                   aafwi_tune_entry *table, int table_cap, int *n_entries,
                   aafwi_plan_opts *best);

/* Number of CUDA kernels this library has launched in this process (a host-
 * side counter incremented at every launch; memsets and copies excluded). */
unsigned long long aafwi_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* AAFWI_H */
