/*
 * dpinn.h - C ABI of libdpinn, a single-GPU (B300, sm_103a) implementation of
 * one training step of the domain-decomposed physics-informed neural network
 * of arXiv 2602.15883 ("Distributed physics-informed neural networks via
 * domain decomposition for fast flow reconstruction"), and of queries on the
 * trained ensemble.
 *
 * Method (paper section / equation numbers count numbered equations in order):
 *   - The space-time box is split into K x M disjoint cells, one independent
 *     fully connected tanh network ("local expert") per cell, mapping
 *     (x, [t]) -> (u, [w], p)                                     Sec. 2.2
 *   - Per net, the local objective (Eq. (16)):
 *       L = l_obs L_obs + l_PDE L_PDE + l_gh_u L_gh_u
 *           + l_space L_gh_p^space + l_time L_gh_p^time
 *     with L_obs (Eq. (3)), L_PDE over the incompressible Navier-Stokes
 *     residuals (Eqs. (5)-(10), 1/Re = nu), the ghost consistency terms
 *     (Eqs. (13)-(14)) against the neighbours' predictions held constant,
 *     the anchor normalisation of the pressure a master sends
 *     (p~ = p(x,t) - p(x_anc,t), Eq. (15)), and l_space = 0 for masters.
 *   - One step (Algorithm 1 with I_comm = 1): neighbour messages at the
 *     current parameters, losses and gradients of every net, then Adam.
 *
 * Readings of the paper used here (where it is silent):
 *   - inputs are mapped from the net's own cell to [-1, 1];
 *   - the ghost set of a net is the union of the points on its shared faces
 *     (one point set per face, used by both sides); L_gh_* of net A divide by
 *     the number of points on all of A's faces, split by face type;
 *   - the anchor is evaluated at each ghost point's own time;
 *   - Adam follows PyTorch (no weight decay); optional per-net clipping
 *     g *= min(1, clip / (||g||_2 + 1e-6)).
 *
 * Conventions
 *   - Every call returns an int status: DPINN_OK (0) or a negative
 *     DPINN_ERR_* code; dpinn_last_error() gives a message.  No C++ exception
 *     crosses the ABI.
 *   - "device pointer" = memory on the handle's GPU; "host pointer" = CPU
 *     memory (pinned or pageable).  Calls that copy accept either (the copy
 *     direction is inferred from the pointer, unified addressing).
 *   - Coordinates are float32 [n][d_in], spatial axes first, time last
 *     (d_in = d_space + unsteady).  Outputs are (u, v, [w], p): d_out =
 *     d_space + 1.
 *   - Nets are numbered over the cell grid with axis 0 fastest:
 *     net = sum_a cell_a * stride_a, stride_0 = 1, stride_a = stride_{a-1} *
 *     splits_{a-1}.  Cell a of a coordinate is decided in float32:
 *     floor((x - (float)lo_a) * (float)(splits_a / (hi_a - lo_a))) clamped to
 *     [0, splits_a - 1] (half-open cells, the last one closed); x outside
 *     [(float)lo_a, (float)hi_a] is outside the domain.
 *   - Faces join net k and k + stride_a for every cell with cell_a <
 *     splits_a - 1; they are numbered axis by axis (ascending), then by k.
 *     A face along the time axis is temporal, all others are spatial.
 *   - Masters are the nets whose spatial cell contains x_anc (one per time
 *     slab).  x_anc is taken at float32 precision.
 *   - Per-net parameter block (the order of get/set_state): for each affine
 *     map l = 0..L (L = depth hidden layers, width W), the weight [out][in]
 *     row-major then the bias [out]; in_0 = d_in, out_L = d_out.
 *   - Loss record of a net: {L_obs, L_PDE, L_gh_u, L_gh_p^space,
 *     L_gh_p^time, L_total} (the spatial pressure term of a master is
 *     reported although its weight is 0).
 */
#ifndef DPINN_H
#define DPINN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dpinn dpinn_t;
/* A cudaStream_t, passed as an opaque pointer (NULL = the legacy stream). */
typedef void* dpinn_stream_t;

enum {
  DPINN_OK = 0,
  DPINN_ERR_INVALID_ARG = -1,
  DPINN_ERR_OOM = -2,
  DPINN_ERR_CUDA = -3,
  DPINN_ERR_NONFINITE = -4,
  DPINN_ERR_TIMEOUT = -5,
  DPINN_ERR_BUSY = -6,
  DPINN_ERR_STATE = -7
};

enum { DPINN_POINTS_RESIDUAL = 0, DPINN_POINTS_OBS = 1, DPINN_POINTS_FACE = 2, DPINN_POINTS_GHOST = 3 };
/* Hidden-layer activation: tanh, or sin (the paper's cylinder cases,
 * Table B1). */
enum { DPINN_ACT_TANH = 0, DPINN_ACT_SIN = 1 };
/* Arithmetic of the hidden-layer contractions of the jet training kernel.
 * FP32: FP32 FMA throughout.  TF32X3 (width 128 only): the three W x W
 * contractions per layer (forward, input adjoint, weight gradient) run on the
 * tcgen05 tensor cores with every FP32 operand split into two TF32 parts and
 * the products accumulated as hi*lo + lo*hi + hi*hi in FP32 (relative error
 * per product ~2^-21, FP32-grade); everything else stays FP32.  In TF32X3
 * the value kernels (observations, ghost terms, messages) and the queries use
 * the same tensor-core arithmetic for their hidden layers, except that the
 * exchange and the face items run the FP32 jet kernels when the interface
 * terms (lambda_gh_r, lambda_gh_c1) are on.  The paper (Sec. 3) trains in
 * FP32 and fixes no kernel arithmetic. */
enum { DPINN_PREC_FP32 = 0, DPINN_PREC_TF32X3 = 1 };

typedef struct dpinn_config {
  int d_space;            /* 2 or 3 */
  int unsteady;           /* 1: time is an input */
  double lo[4], hi[4];    /* global box per input axis */
  int splits[4];          /* cells per input axis */
  int depth;              /* hidden layers L (2..16) */
  int width;              /* neurons per hidden layer: 32, 64, or 128..224
                             (32, 64, 128: register-tiled kernels; 129..224, e.g.
                             the cylinder networks' 150 and 200 of Sec. 5: the
                             streamed-weight kernel, padded to 160 or 224) */
  int activation;         /* DPINN_ACT_TANH or DPINN_ACT_SIN */
  double nu;              /* kinematic viscosity = 1/Re */
  double anchor_x[3];     /* x_anc (spatial) */
  double p_ref;           /* pressure value assigned to x_anc in queries */
  double lambda_obs, lambda_pde, lambda_gh_u;
  double lambda_gh_p_space; /* base value; masters use 0 */
  double lambda_gh_p_time;
  double comp_w[3];       /* velocity component weights in L_obs, L_gh_u */
  double lr, beta1, beta2, eps; /* Adam (PyTorch's rule); beta1, beta2 in [0, 1), else INVALID_ARG */
  double clip_norm;       /* per-net gradient-norm clip, 0 = off */
  uint64_t seed;          /* Xavier-normal initialisation seed */
  int precision;          /* DPINN_PREC_FP32 or DPINN_PREC_TF32X3 */
  int device;             /* CUDA device ordinal */
  /* Step decay of the learning rate (Table B1 "LR factor & interval"): the
   * update of step t (t = 1, 2, ...) uses lr * factor^floor((t-1)/interval);
   * interval 0 = constant lr. */
  double lr_decay_factor;
  int lr_decay_interval;
  /* Communication interval I_comm of Algorithm 1: the neighbour messages
   * are recomputed before step t (t = 0, 1, ... counted before the update)
   * when t mod I_comm == 0 and reused (stale) otherwise.  1 = every step. */
  int comm_interval;
  /* Interface terms beyond C0 continuity (the Remark of Sec. 2.2; the paper
   * leaves them off, 0 = off): residual matching
   *   L_gh_r  = (1/N_gh) sum_ghost ||r_A(x) - sg(r_B(x))||^2  (r: Eqs. (7)-(10))
   * and first-derivative (C1) matching
   *   L_gh_c1 = (1/N_gh) sum_ghost sum_{c,q} (d_q Y_A,c - sg(d_q Y_B,c))^2
   * over every output c (velocity and pressure) and input q, with B the net
   * on the other side (face points) or owning the point (ghost layers);
   * added to L_total with these weights.  Both depend on derivatives only,
   * so no anchor normalisation enters.  When either is > 0 the exchange
   * evaluates jets at the ghost points and the face items train in the FP32
   * jet kernel. */
  double lambda_gh_r, lambda_gh_c1;
} dpinn_config;

typedef struct dpinn_layout {
  int n_nets, n_faces, d_in, d_out, n_params; /* n_params per net */
  int n_masters;
} dpinn_layout;

/* Fill *cfg with defaults (Adam 1e-3 / 0.9 / 0.999 / 1e-8, unit weights,
 * constant lr, I_comm = 1). */
int dpinn_config_default(dpinn_config* cfg);

/* Validate cfg, build the decomposition (cells, faces, masters), allocate
 * all device state on cfg->device and initialise the parameters
 * (Xavier-normal weights from cfg->seed, zero biases).  *out owns everything
 * until dpinn_destroy.  Errors: INVALID_ARG (bad shape, anchor outside the
 * domain, unsupported width/depth), OOM, CUDA. */
int dpinn_create(const dpinn_config* cfg, dpinn_t** out);
void dpinn_destroy(dpinn_t* h);
/* Message of the last failing call on h (h may be NULL for create errors). */
const char* dpinn_last_error(dpinn_t* h);

int dpinn_get_layout(dpinn_t* h, dpinn_layout* out);
/* Master flag and cell box (lo[4], hi[4], unused axes 0) of net k. */
int dpinn_net_info(dpinn_t* h, int net, int* is_master, double* lo4, double* hi4);
/* Nets on the low / high side of face f, its axis and 1 if temporal. */
int dpinn_face_info(dpinn_t* h, int face, int* net_lo, int* net_hi, int* axis, int* is_time);

/* Deliver a point set (copied into handle-owned device memory).
 *   kind RESIDUAL: pts [n][d_in], counts[n_nets] (points of net 0 first).
 *   kind OBS:      pts [n][d_in], vals [n][d_space] (observed velocity),
 *                  counts[n_nets].
 *   kind FACE:     pts [n][d_in], counts[n_faces] (points of face 0 first;
 *                  each point must lie on its face).
 *   kind GHOST:    pts [n][d_in], counts[n_nets]: the paper's volumetric
 *                  ghost layers (Sec. 2.2, thickness delta > 0): net A's
 *                  points lie in its cell grown by delta, outside the cell
 *                  itself.  Each point is routed (float32 rule) to the net B
 *                  whose cell holds it - corner regions reach diagonal
 *                  neighbours - and A's ghost terms compare against B's
 *                  prediction there (anchor-normalised when B is a master).
 *                  The pressure term is temporal when A and B share their
 *                  spatial cell, spatial otherwise.  Replaces FACE points
 *                  (delivering FACE points switches back).  A point inside
 *                  A's own cell or outside the domain is INVALID_ARG.
 * pts/vals may be host or device pointers.  n_counts must equal n_nets (or
 * n_faces).  Counts may be 0.  Re-delivering the same counts only copies;
 * new counts rebuild the work lists and the captured step.  Errors:
 * INVALID_ARG, OOM, CUDA. */
int dpinn_set_points(dpinn_t* h, int kind, const float* pts, const float* vals,
                     const int64_t* counts, int n_counts);

/* Self-test of failure detection (no counterpart in the paper): runs a
 * one-block kernel that waits, with the same bounded wait the kernels use
 * for their copies and MMAs, on an mbarrier that nothing ever completes.
 * Expected result: DPINN_ERR_TIMEOUT after about 2 s; the kernel returns
 * normally, so the CUDA context and the handle stay usable (the handle's own
 * error words are not touched).  STATE if the wait returned without giving
 * up.  Synchronises the device. */
int dpinn_selftest_wait(dpinn_t* h);

/* Self-test of the sine and cosine that the sin-activation kernels evaluate
 * (the activation of the paper's cylinder networks; the evaluation itself
 * has no counterpart in the paper): out[2 i] = sin x[i], out[2 i + 1] =
 * cos x[i], computed exactly as the kernels do (a Cody-Waite reduction by
 * pi/2 in three parts and Taylor series on [-pi/4, pi/4]; within a few ulp
 * for |x| < 6400, NaN for NaN and infinite x).  x: n floats, out: 2 n
 * floats, both device memory on `device`, owned by the caller.  n = 0 is a
 * no-op.  Synchronises.  Errors: INVALID_ARG (n < 0, or null pointers with
 * n > 0), CUDA. */
int dpinn_selftest_sincos(int device, const float* x, long long n, float* out);

/* Asynchronous upload of the residual points for the next step/* Asynchronous upload of the residual points for the next step (same
 * counts as the current set; other layouts fall back to dpinn_set_points).
 * The host -> device copy runs on an internal stream into a staging buffer,
 * overlapping the work already queued; the next dpinn_step / dpinn_eval_*
 * waits for it on its own stream and moves the points into place (a
 * device-to-device copy) before its kernels.  `pts` (pinned host memory for
 * a true overlap) must stay unchanged until that next call has been issued
 * and its work has completed.  One upload may be pending at a time.
 * `stream` is unused (reserved).  Errors: INVALID_ARG (kind other than
 * RESIDUAL, counts length), STATE (an upload already pending), CUDA. */
int dpinn_set_points_async(dpinn_t* h, int kind, const float* pts, const int64_t* counts, int n_counts,
                           dpinn_stream_t stream);

/* Per-step resampling of the collocation points/* Per-step resampling of the collocation points (mini-batch epochs: fresh
 * residual points every step, none stored or copied from the host).  The
 * paper trains on fixed point sets per epoch (Sec. 3, Table B1); this call,
 * which the paper has no counterpart of, draws counts[k] points uniformly in
 * net k's interior cell before each training step, losses-only or gradient
 * evaluation, on the device.  Generator (counter-based, reproducible): with
 * mix the output function of SplitMix64 (Steele, Lea, Flood 2014:
 * z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
 * z ^= z >> 31) and gamma = 0x9E3779B97F4A7C15, all modulo 2^64,
 *   S_t     = mix(seed + (t + 1) gamma)      t = steps taken so far
 *   S_{t,k} = mix(S_t + (k + 1) gamma)
 *   u       = (mix(S_{t,k} + (i d_in + d + 1) gamma) >> 40) * 2^-24
 *   x_{i,d} = (float)(lo_{k,d} + u * (hi_{k,d} - lo_{k,d}))   (double, no FMA)
 * for point i (0-based within net k) and input axis d, where lo/hi are the
 * cell bounds lo_d + c_d (hi_d - lo_d) / splits_d in double.  counts [n_nets]
 * (host); counts == NULL switches resampling off and keeps the last sampled
 * set as the residual points.  dpinn_set_points(RESIDUAL) also switches it
 * off.  Errors: INVALID_ARG (length, negative count, more than 2^30 points),
 * CUDA. */
int dpinn_set_resampling(dpinn_t* h, const int64_t* counts, int n_counts, uint64_t seed);

/* Synchronise and copy the current points of a set (kind RESIDUAL, OBS or
 * FACE; [n][d_in] float32, n = the sum of that set's counts) to host_out.
 * With resampling, the residual points are those of the most recent step or
 * evaluation.  Errors: INVALID_ARG, STATE (set not present), CUDA. */
int dpinn_get_points(dpinn_t* h, int kind, float* host_out);

/* Memory budget (bytes, 0 = the default of 1 GiB) for the per-work-item
 * gradient partials: the plan enlarges its point chunks until
 * (number of items) x (per-net parameter stride) x 4 bytes fits, so the
 * number of points per step is not limited by this memory.  The gradient is
 * the same sum, in a different (fixed) order.  Rebuilds the plan. */
int dpinn_set_partial_budget(dpinn_t* h, int64_t bytes);

/* Run n_steps training iterations asynchronously on `stream` (one captured/* Run n_steps training iterations asynchronously on `stream` (one captured
 * CUDA graph per step: exchange, losses + gradients of all nets, Adam).
 * Errors: STATE (points missing), CUDA. */
int dpinn_step(dpinn_t* h, dpinn_stream_t stream, int n_steps);

/* Like one step without the optimiser update: losses and gradients at the
 * current parameters; the gradient is readable with dpinn_get_grad. */
int dpinn_eval_grad(dpinn_t* h, dpinn_stream_t stream);

/* Losses only (no reverse pass, no update) at the current parameters, on
 * `stream`; read them with dpinn_loss. */
int dpinn_eval_loss(dpinn_t* h, dpinn_stream_t stream);

/* Replace the parameters ([n_nets][n_params], host or device pointer)
 * without touching the Adam moments or the step count.  Synchronises. */
int dpinn_set_params(dpinn_t* h, const float* params);

/* Synchronise with the handle's work and copy the loss record of the most
 * recent step (evaluated at its pre-update parameters) to host_out
 * [n_nets][6].  Errors: NONFINITE (a loss is NaN/Inf; host_out still
 * filled), TIMEOUT (a device wait gave up), CUDA. */
int dpinn_loss(dpinn_t* h, float* host_out);

/* Asynchronous form of dpinn_loss for pipelined training loops: enqueue on
 * `stream`, after the work already queued there, a copy of the loss record
 * [n_nets][6] into host_out and return without waiting.  The caller owns
 * host_out (pinned host memory, else the copy is synchronous); its contents
 * are valid once `stream` has reached this point (an event recorded after
 * the call).  Call it on the stream the step ran on, before the next step
 * is queued there, which overwrites the record.  The device error flags are
 * not read: NONFINITE and TIMEOUT stay set and are reported by the next
 * dpinn_loss / dpinn_loss_ext.  Errors: INVALID_ARG, CUDA. */
int dpinn_loss_async(dpinn_t* h, float* host_out, dpinn_stream_t stream);

/* As dpinn_loss with the 8-entry record [n_nets][8]: the 6 entries above
 * (the total includes the interface terms), then L_gh_r and L_gh_c1. */
int dpinn_loss_ext(dpinn_t* h, float* host_out);

/* Gradient of the most recent step or dpinn_eval_grad (before clipping),
 * out [n_nets][n_params] in the parameter-block order (host or device
 * pointer).  Synchronises. */
int dpinn_get_grad(dpinn_t* h, float* host_out);

/* Query the resident ensemble: route each point to its cell, evaluate the
 * net.  out row = (u, v, [w], p_out) or, with want_residual, followed by the
 * d_space + 1 residuals (momentum then continuity; the raw-pressure
 * gradient enters them).  p_out = p - p(x_anc, t) + p_ref in master cells,
 * p + p_ref elsewhere (Eq. (18)).  pts [n][d_in] and out [n][row] are device
 * pointers owned by the caller; asynchronous on `stream`.  A point outside
 * the domain sets an error that the next dpinn_query_status reports
 * (INVALID_ARG); its row is left untouched. */
int dpinn_query(dpinn_t* h, const float* dev_pts, int64_t n, int want_residual,
                float* dev_out, dpinn_stream_t stream);
/* Output jets of the nets at routed points: for each point, the jets of the
 * net whose cell holds it, row [j][c] of d_out x (d_in + 2) floats - outputs
 * j = (u, v, [w], p), channels c = value, d/dx_q for every input q (spatial
 * axes, then time), spatial Laplacian.  These are the forward jets the
 * residuals of Eqs. (7)-(10) are assembled from (value, first derivatives and
 * Laplacian carried through the network of Eq. (2), Sec. 2.1).  The pressure
 * is the net's raw output (no anchoring, no p_ref).  Same kernels, routing,
 * ownership, asynchrony and error reporting as dpinn_query with
 * want_residual = 1; pts [n][d_in] and out [n][d_out][d_in + 2] are device
 * pointers owned by the caller.  Errors: INVALID_ARG (n < 0 or > 2^30, null
 * pointers), OOM, CUDA; points outside the domain as for dpinn_query. */
int dpinn_query_jets(dpinn_t* h, const float* dev_pts, int64_t n, float* dev_out, dpinn_stream_t stream);

/* Query contexts: dpinn_query shares one scratch per handle, so two of its
 * calls must not overlap on the GPU.  A context owns its own routing scratch
 * for up to max_points points per call (one device allocation made here, of
 * about 8.5 bytes per point plus 44 bytes per net) and its own error words,
 * so queries through different contexts may run concurrently
 * on different streams (the serving loop keeps one per in-flight batch).
 * dpinn_qctx_query: as dpinn_query (device pointers, asynchronous on
 * `stream`); n > max_points is INVALID_ARG.  dpinn_qctx_status: synchronise
 * `stream`, report (then clear) the context's out-of-domain error.  A
 * context must be destroyed before its handle. */
typedef struct dpinn_qctx dpinn_qctx_t;
int dpinn_qctx_create(dpinn_t* h, int64_t max_points, dpinn_qctx_t** out);
void dpinn_qctx_destroy(dpinn_qctx_t* q);
int dpinn_qctx_query(dpinn_qctx_t* q, const float* dev_pts, int64_t n, int want_residual,
                     float* dev_out, dpinn_stream_t stream);
int dpinn_qctx_status(dpinn_qctx_t* q, dpinn_stream_t stream);

/* Same as dpinn_query, for callers that must not allocate device memory
 * while serving: a latency-bound loop that cannot afford the device-wide
 * synchronisation a cudaMalloc implies, or code whose device memory is owned
 * by another framework's allocator.  dpinn_query grows handle-owned scratch
 * with cudaMalloc when a request is larger than any before it; this variant
 * calls no cudaMalloc, cudaFree or allocating library routine.  Its scratch
 * is one fixed array in device memory (about 2.4 MB) that every GPU loading
 * this library holds until the process exits.  (The paper has no
 * counterpart: this is a serving convenience.)
 *   - n <= 262144 points per call and at most 4096 nets, else INVALID_ARG
 *     with a message; pts/out are device pointers owned by the caller.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device made current); make that first call
 *     before any stream capture.  The address is kept for the life of the
 *     process: it does not survive a device reset.
 *   - A request whose work items would not fit the array is refused with
 *     STATE before anything is launched (cannot happen with the kernels of
 *     this library, whose query tiles have at least 16 points).
 *   - All calls share the one array and leave their contents in it; each
 *     call clears what must start at zero.  Calls that overlap on the GPU
 *     (different streams, or several handles on one device) race on it:
 *     issue them on one stream or serialise them.
 *   - Errors of points outside the domain are reported by
 *     dpinn_query_status, as for dpinn_query. */
int dpinn_query_static(dpinn_t* h, const float* dev_pts, int64_t n, int want_residual,
                       float* dev_out, dpinn_stream_t stream);

/* Synchronise `stream` and report (then clear) out-of-domain errors. */
int dpinn_query_status(dpinn_t* h, dpinn_stream_t stream);

/* Parameters, Adam moments and step count, host buffers of
 * [n_nets][n_params] floats (any pointer may be NULL to skip it). */
int dpinn_get_state(dpinn_t* h, float* params, float* m, float* v, int64_t* step);
int dpinn_set_state(dpinn_t* h, const float* params, const float* m, const float* v,
                    int64_t step);

/* Apply one optimiser update with a given gradient (host [n_nets][n_params]);
 * the same kernels as the step's update. */
int dpinn_apply_grad(dpinn_t* h, const float* host_grad);

/* Schedule of the grouped kernels: points per work item of the jet (residual)
 * and value (observation / face) kernels, in tiles of their tile size
 * (0 = automatic: about 8 items per SM, at most 64 tiles), and the order in
 * which the persistent CTAs take items (0 = longest first, 1 = net order).
 * Rebuilds the work lists and recaptures the step; results do not depend on
 * the schedule beyond float rounding of the gradient sums (each schedule is
 * itself deterministic).  Used by the autotuner. */
int dpinn_set_schedule(dpinn_t* h, int jet_tiles, int val_tiles, int order);
/* Switch the arithmetic of the hidden-layer contractions (DPINN_PREC_FP32 or
 * DPINN_PREC_TF32X3, the latter for width 128 only) on a live handle: the
 * step, the value items and the queries then launch the other kernel family
 * (the same work, Eqs. (2)-(16) and Algorithm 1; both meet the same error
 * bounds against FP64).  Parameters, Adam moments, step count and points are
 * kept; the work lists and the captured step are rebuilt for the new kernels'
 * tiles.  Synchronises the device.  Used by the autotuner, which times both
 * and keeps the faster.  Errors: INVALID_ARG (unknown precision, TF32X3 at
 * another width), CUDA, OOM.  dpinn_get_precision reports the current one. */
int dpinn_set_precision(dpinn_t* h, int precision);
int dpinn_get_precision(dpinn_t* h, int* precision);

/* Register tiles of the grouped kernels.  dpinn_tile_options lists, for the
 * current precision, the tiles available for the jet training kernel and for
 * the value kernels (observation / ghost training and the exchange) as their
 * sizes in points, default first: up to 2 each (the FP32 kernels are
 * instantiated with a default and an alternate register tile - at width 128
 * with jets the alternate keeps the 16-point tile with 8 neurons x 1 point
 * per thread instead of 4 x 2, so two options can have the same size; the
 * tensor-core kernels have one).  dpinn_set_tiles selects them by index into
 * those lists (0 = the default); the work lists and the captured step are
 * rebuilt, results are the same up to float rounding of the gradient sums.
 * dpinn_get_tiles reports the indices in use.  Used by the autotuner.
 * Errors: INVALID_ARG (an index not offered), CUDA, OOM. */
int dpinn_tile_options(dpinn_t* h, int* jet_points, int* n_jet, int* val_points, int* n_val);
int dpinn_set_tiles(dpinn_t* h, int jet_tile, int val_tile);
int dpinn_get_tiles(dpinn_t* h, int* jet_tile, int* val_tile);

/* Current schedule and the tile sizes (points) of the jet and value kernels
 * (tile_points[2]). */
int dpinn_get_schedule(dpinn_t* h, int* jet_tiles, int* val_tiles, int* order, int* tile_points);

/* Kernels launched by one dpinn_step (for accounting). */
int dpinn_launches_per_step(dpinn_t* h);

/* One training step (identical kernels and launch configuration to
 * dpinn_step, launched individually instead of as a graph) with a CUDA event
 * recorded on `stream` around every kernel.  Synchronises; writes up to
 * max_kernels durations (ms) to ms[], their count to *n_kernels and static
 * kernel names to names[] (may be NULL). */
int dpinn_step_timed(dpinn_t* h, dpinn_stream_t stream, float* ms, int max_kernels, int* n_kernels,
                     const char** names);

/* Measurement aid (not part of the training path): time one launch of a
 * kernel in which every thread runs 8 independent chains of packed dual
 * FP32 FMAs (blocks_per_sm x 256-thread CTAs per SM, `iters` iterations of
 * 32 packed FMAs per thread) on `device`, after a short warm-up launch.
 * Returns the launch time in *ms (CUDA events) and its FLOP count in *flop;
 * *flop / *ms is the attainable FP32 FMA rate at the clocks the GPU ran.
 * Synchronises.  Errors: INVALID_ARG (blocks_per_sm outside 1..8, iters
 * outside 1..2^40, null outputs), CUDA. */
int dpinn_probe_fp32(int device, int blocks_per_sm, long long iters, float* ms, double* flop);

#ifdef __cplusplus
}
#endif
#endif /* DPINN_H */
