/*
 * libasicp: GB300 (sm_103a) implementation of the data-parallel hot path of
 * Annealed Stein ICP (AS-ICP) grasp matching, from "Grasping by Parallel Shape
 * Matching" (arXiv 2412.08346).  For every gripper preshape and every pose
 * particle it transforms the gripper contact cloud, finds nearest-neighbour
 * correspondences in the object cloud, evaluates the cost and gradient of the
 * paper's loss (matching term, TCP-CoM term, SDF collision term) and applies
 * the annealed SVGD / SGD-ICP update (Algorithm 1).
 *
 * Conventions for every call below
 *  - Units are metres in the object frame (Section IV-A).  A pose is
 *    theta = (t_x, t_y, t_z, q_w, q_x, q_y, q_z): a translation and a unit
 *    quaternion, scalar first (Section III-A).  Point arrays are packed xyz
 *    float32 triples, row-major.
 *  - Input and output arrays may live in host memory (pageable or pinned) or in
 *    device memory of the context's GPU; the library tells them apart through
 *    unified addressing.  The caller keeps ownership; the library copies what it
 *    keeps, so an input may be freed or reused as soon as the call returns.
 *  - All device work is issued on asicp_config.cuda_stream (NULL: the legacy
 *    default stream).  Calls that produce host-visible results
 *    (asicp_best_grasps, asicp_get_state, asicp_kernel_times) and the input
 *    calls that validate their data (asicp_set_object, asicp_set_gripper_sdf)
 *    synchronise that stream; asicp_step and asicp_run only enqueue work.
 *  - Errors are returned as asicp_status; no C++ exception crosses this
 *    boundary.  A failing call leaves the context valid and records a message
 *    readable with asicp_last_error.  A context is not thread-safe: use one
 *    context per host thread.
 */
#ifndef ASICP_H
#define ASICP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct asicp_ctx asicp_ctx;

typedef enum {
    ASICP_OK = 0,
    ASICP_ERR_INVALID_ARG = 1, /* bad pointer, size, index or non-finite input value      */
    ASICP_ERR_STATE = 2,       /* call order: e.g. asicp_step before the inputs are set   */
    ASICP_ERR_CUDA = 3,        /* a CUDA runtime call or a kernel launch failed            */
    ASICP_ERR_OOM = 4,         /* device or host allocation failed                         */
    ASICP_ERR_TIMEOUT = 5      /* a bounded device-side wait expired                       */
} asicp_status;

/* Parameters of Algorithm 1.  asicp_config_default fills Table I's values and the
 * readings the paper leaves open:
 *   P, K          preshapes and particles per preshape (K <= 1024)
 *   k_max, k_stein total iterations and SVGD iterations (Algorithm 1; Table I
 *                  gives 15 SVGD + 25 SGD, default k_stein = round(0.375 k_max))
 *   schedule      0: cyclic annealing gamma = (mod(k, k_max/C) / (k_max/C))^p
 *                  (Eq. 11, Table I: C = 5, p = 2); 1: linear g0 -> g1
 *   eta_sgd       SGD-ICP learning rate (Eq. 3, Table I: 1); the preconditioner A is I
 *   eta_svgd      SVGD step (Eq. 7); <= 0 selects 1/N
 *   w_com         weight of the TCP-CoM term inside the 1/N of Eqs. 16-17 (Table I: 1)
 *   bandwidth_mode 0: median heuristic h = med_{i<j}|t_i - t_j|^2 / ln K; 1: h_fixed (Eq. 9)
 *   conv_tol      relative cost change that freezes a particle in the SGD phase
 *                  (Section IV-D, Table I: 0.02 %); < 0 disables freezing
 *   init_radius   radius of the Fibonacci-sphere initial poses around the CoM (Section V)
 *   debug         1: keep per-query correspondences, transformed points and collision
 *                  lists so asicp_get_state can return them (costs memory and bandwidth)
 *   profile       1: time the main kernels with CUDA events (asicp_kernel_times);
 *                  2: time the forward-matching (screening) kernel only.  The events
 *                  are nodes of the captured iteration loop and add a few
 *                  microseconds each to a pass (profile 1: ~5 % of a paper-scale
 *                  grasp set on GB300)
 *   cuda_stream   cudaStream_t for all work, NULL for the default stream
 *   n_objects     objects optimised together in one pass (one grasp set each, default 1);
 *                  every kernel covers all of them, each particle matched against its
 *                  own object (Section IV-D's "combine into multidimensional tensors",
 *                  extended across objects)
 *   autotune      1: the first asicp_run times the forward-matching kernel shapes on its
 *                  workload and keeps the fastest (see asicp_autotune); 0: use fwd_shape
 *   fwd_shape     forward-matching kernel shape, 0 .. ASICP_FWD_SHAPES-1 (0 = default):
 *                  0 .. ASICP_FWD_SHAPES-2 are float32 kernels, ASICP_FWD_SHAPES-1 the
 *                  tensor-core screening with its exact-choice kernel (not with mini-batches).
 *                  Every shape returns the lowest-index minimum of the exact-form float32
 *                  distance over the points that can be nearest; they can differ only where
 *                  several points' float32 distances tie within rounding (near-ties)
 *   init_mode     initial poses when asicp_run gets none: 0 = Fibonacci sphere of radius
 *                  init_radius around the CoM, approach axis towards the CoM; 1 = the
 *                  variant of the paper's experiments (Section VI-A, Fig. 3 (b)):
 *                  Fibonacci points on the quarter of the sphere facing the robot (z >= 0,
 *                  x >= 0 relative to the CoM; spiral z_j = 1 - (j + 1/2)/n, azimuth
 *                  (j golden angle mod pi) - pi/2) plus min(6, K_g) poses directly above
 *                  the object, approach axis -z, yawed 0, 60, ..., 300 degrees
 *   prior_t_sigma, prior_q_kappa, prior_q_mean
 *                 the priors of Eq. 8 (Section IV-A: Gaussian on translations, von Mises on
 *                  rotations), used in the SVGD phase: the drive of particle j becomes
 *                  gamma (-N g_j + grad log p(theta_j)) with grad_t log p = -(t - CoM) /
 *                  prior_t_sigma^2 and grad_q log p = prior_q_kappa sign(mu.q) mu, mu =
 *                  prior_q_mean normalised (q and -q alike); 0 switches a prior off (the
 *                  default: the paper gives no parameters)
 * Particles are numbered object by object, preshape by preshape: the group
 * g = object * P + preshape holds K_g particles (K_g = K unless set with
 * asicp_set_particle_counts); T = sum of K_g is the particle count of every
 * per-particle array below. */
#define ASICP_FWD_SHAPES 8

typedef struct {
    int P, K;
    int k_max, k_stein;
    int schedule;
    float C_cycles, p_exp, g0, g1;
    float eta_sgd, eta_svgd;
    float w_com;
    int bandwidth_mode;
    float h_fixed;
    float conv_tol;
    float init_radius;
    int debug;
    int profile;
    void *cuda_stream;
    int n_objects;
    int autotune;
    int fwd_shape;
    int init_mode;
    float prior_t_sigma, prior_q_kappa;
    float prior_q_mean[4];
} asicp_config;

/* Host pointers (or device pointers) the library fills in asicp_get_state; any
 * may be NULL.  T = total particle count; with one object and uniform K the flat
 * particle index is p * K + j.
 *   theta     T*7 float     poses (after the last step's update)
 *   cost      T   double    cost at the poses the last step started from: the match
 *                           cost L (Eqs. 13-15) or, for a colliding particle, L_col (Eq. 18)
 *   grad      T*7 double    gradient used by the last step (Eqs. 16-17, or Eq. 18 via 4-5)
 *   phi       T*7 float     Stein direction of the last step (Eq. 8; zero in the SGD phase)
 *   ncol      T   int       colliding points of C at those poses (Eq. 12)
 *   frozen    T   int       convergence flag
 *   h         G   float     RBF bandwidth of every group in the last SVGD step (Eq. 9)
 * needing config.debug = 1:
 *   nn_idx    T*N int       forward correspondence index into R per gripper point (Eq. 1)
 *   nn_d2     T*N float     its squared distance
 *   s_prime   T*N*3 float   transformed gripper points exactly as matched
 *   col_list  sum over particles of their object's Mc, int: for every particle, Mc
 *                           entries (object by object, particle by particle); the first
 *                           ncol hold the colliding C indices, ascending
 *   col_nn    same layout   nearest gripper point per colliding point (Eq. 18)     */
typedef struct {
    float *theta;
    double *cost;
    double *grad;
    float *phi;
    int *ncol;
    int *frozen;
    float *h;
    int *nn_idx;
    float *nn_d2;
    float *s_prime;
    int *col_list;
    int *col_nn;
} asicp_state_view;

/* Fill *cfg with the defaults described above for P = 1, K = 32, k_max = 40, one object. */
void asicp_config_default(asicp_config *cfg);

/* Create a context for one GPU (the current device).  *out receives the handle.
 * Errors: INVALID_ARG for NULL pointers or out-of-range parameters, OOM. */
asicp_status asicp_create(const asicp_config *cfg, asicp_ctx **out);

/* Release every device and host resource of ctx (NULL is accepted). */
asicp_status asicp_destroy(asicp_ctx *ctx);

/* Object cloud R (M x 3) used for matching (Eq. 1, the reference cloud R of
 * Section III-A) and collision cloud C (Mc x 3; object and table, Section IV-A).
 * C_xyz = NULL uses C = R.  Computes CoM = centroid of R (Algorithm 1).  A new
 * object with the same M and Mc as the previous one keeps the context's layout,
 * its poses and its captured iteration loop; other sizes need new poses
 * (asicp_set_state or asicp_run) before asicp_step.  Mini-batches set with
 * asicp_set_minibatch are dropped.
 * Errors: INVALID_ARG (NULL R, M < 1, Mc < 1 when C is given, non-finite value). */
asicp_status asicp_set_object(asicp_ctx *ctx, const float *R_xyz, int M, const float *C_xyz, int Mc);

/* The same for object `object` (0 <= object < n_objects); objects may have
 * different M and Mc.  Errors: as asicp_set_object, INVALID_ARG for the index. */
asicp_status asicp_set_object_at(asicp_ctx *ctx, int object, const float *R_xyz, int M, const float *C_xyz, int Mc);

/* Particles per group: K[object * P + preshape], n = n_objects * P values in
 * [1, 1024].  Clears the poses.  Errors: INVALID_ARG. */
asicp_status asicp_set_particle_counts(asicp_ctx *ctx, const int *K, int n);

/* Preshape `preshape` (0 <= preshape < P): contact-surface cloud S (N x 3, gripper
 * frame; the source cloud of Section IV-A) and the gripper's signed distance field
 * sampled on a node-centred grid of nx*ny*nz float32 values, x fastest, positive
 * inside the gripper (Eq. 12), node (0,0,0) at origin, spacing voxel.  Computes
 * TCP = centroid of S (Section IV-B).  Every preshape must have the same N
 * (1 <= N <= 6144).  The context keeps a copy of the grid and a corner-packed
 * copy for the lookups (32 bytes per cell: 8 (nx-1)(ny-1)(nz-1) floats).
 * Errors: INVALID_ARG (index, N out of range, a grid dimension < 2, voxel <= 0, N differing
 * from an earlier preshape, non-finite value). */
asicp_status asicp_set_gripper_sdf(asicp_ctx *ctx, int preshape, const float *S_xyz, int N,
                                   const float *sdf, int nx, int ny, int nz,
                                   const float origin[3], float voxel);

/* Set all T poses (T*7 floats; quaternions are normalised) and the iteration
 * counter, clearing the convergence state.  Used for warm starts and to
 * teacher-force a single step.  Errors: INVALID_ARG, STATE (inputs not set). */
asicp_status asicp_set_state(asicp_ctx *ctx, const float *theta, int k);

/* Set the convergence state that the next SGD-phase step reads (Table I's
 * convergence criterion, Section IV-D): prev_cost[T] (float64; the cost of the
 * previous iteration, negative = none) and frozen[T] (int; nonzero = converged,
 * the SGD update skips the particle).  In the SGD phase a step freezes a particle
 * whose relative cost change |L_k - L_(k-1)| / L_(k-1) is at most conv_tol and
 * unfreezes every particle with a colliding point; every step then stores its
 * cost as the next previous cost.  Call after asicp_set_state (which clears
 * both) to resume or teacher-force a step; either pointer may be NULL (that part
 * is kept).  Host or device pointers, copied.  Errors: STATE (poses not set),
 * CUDA. */
asicp_status asicp_set_convergence(asicp_ctx *ctx, const double *prev_cost, const int *frozen);

/* One iteration k (0 <= k < k_max) of Algorithm 1 for all preshapes and
 * particles: transform, match, cost/gradient, collision test and collision
 * gradient, then the SVGD update (k < k_stein, Eqs. 7-11) or the SGD-ICP update
 * (Eq. 3).  Errors: STATE (inputs or poses not set, or sizes changed since the
 * poses were set), INVALID_ARG (k), CUDA. */
asicp_status asicp_step(asicp_ctx *ctx, int k);

/* Full optimisation of every object's grasp set: initial poses theta0 (T*7,
 * normalised here) or, for theta0 = NULL, for every group the Fibonacci sphere of
 * K_g poses of radius init_radius around its object's CoM (Section V); k_max steps;
 * a final evaluation of cost and collisions at the last poses; and the per-object
 * ranking used by asicp_best_grasps (Algorithm 1's argmin).  The loop is replayed
 * from a captured CUDA graph.  Errors: STATE, INVALID_ARG, CUDA. */
asicp_status asicp_run(asicp_ctx *ctx, const float *theta0);

/* The topk best particles of object 0 in the last asicp_run: non-colliding first,
 * then by ascending final cost, ties to the lower flat index.  theta: topk*7
 * floats, cost: topk floats, preshape: topk ints (any may be NULL); *n_out =
 * entries written (min(topk, particles of the object)).
 * Errors: STATE (no completed run), INVALID_ARG. */
asicp_status asicp_best_grasps(asicp_ctx *ctx, int topk, float *theta, float *cost, int *preshape, int *n_out);

/* The same for object `object`.  Errors: as asicp_best_grasps, INVALID_ARG for the index. */
asicp_status asicp_best_grasps_at(asicp_ctx *ctx, int object, int topk, float *theta, float *cost, int *preshape,
                                  int *n_out);

/* Copy the current particle state into the arrays of *view (see above).
 * Errors: STATE (debug arrays requested without config.debug, or no step yet). */
asicp_status asicp_get_state(asicp_ctx *ctx, const asicp_state_view *view);

/* With config.profile = 1: accumulated device time (ms) and launch count of the
 * path's kernels since the last reset (profile = 2: the forward-matching entry
 * only, the others stay 0).  ms[ASICP_KERNEL_KINDS] / launches[...]
 * order: forward matching (screening; with the float32 shapes also the exact
 * choice), collision test (with the matching sums), reverse matching, finalize
 * (cost, gradient, convergence, SGD step), Stein (SVGD step: the Stein direction
 * and the update kernel, timed and counted together as one launch per pass), and
 * the exact choice of the tensor-core shape (no launches with the float32
 * shapes).  reset = 1 clears the counters after reading.  Errors: STATE (profile
 * off). */
#define ASICP_KERNEL_KINDS 6
asicp_status asicp_kernel_times(asicp_ctx *ctx, double ms[ASICP_KERNEL_KINDS], long long launches[ASICP_KERNEL_KINDS],
                                int reset);

/* Forward matching without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory, such as
 * real-time control loops that reserve all memory at start-up and cannot afford the
 * device synchronisation of cudaMalloc/cudaFree, or runtimes that hand out all
 * device memory from their own pool.  It computes what asicp_step's matching stage
 * computes: for every particle p*K+j and gripper point i, the index of the nearest
 * object point, ties to the lowest index, written to nn_idx[(p*K + j)*N + i].
 *   theta   P*K*7 floats (poses, quaternions are normalised), S_xyz P*N*3 floats
 *           (gripper clouds, preshape-major), R_xyz M*3 floats: host or device memory
 *           (host inputs are staged through the scratch array, not allocated)
 *   nn_idx  P*K*N int32 output, device memory
 *   cuda_stream  cudaStream_t (NULL: default stream); the call waits for the stream
 *           twice (after checking the inputs and at the end) and returns when nn_idx
 *           is written
 * Its scratch is one fixed-size static device array (5 MiB) that every device that
 * loads the library keeps until the process exits; it bounds the sizes to
 * P*K <= ASICP_NOALLOC_MAX_PK, P*N <= ASICP_NOALLOC_MAX_PN, M <= ASICP_NOALLOC_MAX_M
 * (larger problems: use the context API).  The first call on a device looks the
 * array's device address up once (make it before any stream capture).  All calls
 * share the array: calls that overlap on the GPU race and must be ordered by the
 * caller.  Returns INVALID_ARG for NULL pointers, sizes < 1 or beyond the limits,
 * nn_idx not in device memory, or a non-finite input (nn_idx is then left
 * untouched); TIMEOUT if a bounded device wait expired (nn_idx undefined); CUDA for
 * a failed CUDA call. */
#define ASICP_NOALLOC_MAX_PK 16384
#define ASICP_NOALLOC_MAX_PN 65536
#define ASICP_NOALLOC_MAX_M 65536
asicp_status asicp_match_noalloc(const float *theta, int P, int K, const float *S_xyz, int N,
                                 const float *R_xyz, int M, int *nn_idx, void *cuda_stream);

/* Mini-batches of the object cloud for the matching (Eq. 14 and Table I: iteration
 * k matches the gripper points against a mini-batch of R whose size ramps up, N
 * min(k, 2 k_max/3) / (2 k_max/3) in Table I).  offsets [iters + 1] (offsets[0] = 0)
 * and indices [offsets[iters]] give per iteration k < iters the mini-batch as
 * ascending indices into R; iterations k >= iters, and the final evaluation of
 * asicp_run, use the whole cloud.  The collision test, the CoM and the cost
 * normalisation (by N) keep the whole object; with debug = 1 the correspondences
 * read back are positions within the mini-batch.  Host or device pointers, copied;
 * NULL offsets switch mini-batches off; asicp_set_object switches them off too.
 * One object per context; not with the tensor-core kernel shape (7), which the
 * autotuner then skips.  Errors: INVALID_ARG (sizes, ranges, order, n_objects > 1),
 * STATE (no object), CUDA. */
asicp_status asicp_set_minibatch(asicp_ctx *ctx, const int *offsets, const int *indices, int iters);

/* Time every shape of the forward-matching kernel (queries per thread, screening
 * chunk, threads per CTA, shared-memory tile size) on the context's current
 * objects and poses (the Fibonacci initial poses when none are set) and keep the
 * fastest for later steps and runs.  *chosen receives the shape index
 * (0 .. ASICP_FWD_SHAPES-1), ms[ASICP_FWD_SHAPES] the mean launch time of each
 * shape (either may be NULL).  The shapes differ in speed; their results agree
 * up to near-ties (see config.fwd_shape).  With a mini-batch ramp set, the
 * tensor-core shape is skipped (its ms entry is 0).
 * Errors: STATE (inputs not set), CUDA. */
asicp_status asicp_autotune(asicp_ctx *ctx, int *chosen, float *ms);

/* Testing aid for the bounded-wait path.  Every device-side wait of the library
 * is bounded (2^32 SM clock cycles, about 2 s); when one expires, the kernel sets
 * the context's error word, drains its copies in flight with the full budget and
 * returns, the later kernels of the pass see the error word and skip their work,
 * and the next call that reads results (asicp_get_state, asicp_best_grasps)
 * returns TIMEOUT and clears the word; the context stays usable.  With on != 0 the
 * float32 matching shapes' kernels of later asicp_step / asicp_run calls make each
 * CTA's first copy wait on an mbarrier that nothing arrives at, for 1000 cycles,
 * so that it expires; on = 0 restores normal waits (a captured loop is
 * re-captured).  The tensor-core shape ignores it.  Errors: none beyond a NULL
 * context. */
asicp_status asicp_test_expire_waits(asicp_ctx *ctx, int on);

/* Message of the last failing call on ctx (owned by ctx, valid until its next call). */
const char *asicp_last_error(const asicp_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
