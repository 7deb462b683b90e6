/*
 * grid.h -- C-ABI of the GB300-native rigid-body dynamics library.
 *
 * The library computes, for N independent knot points of a trajectory, the
 * algorithms of Sec. IV-B of the GRiD paper (Plancher et al., arXiv 2109.06976):
 * inverse dynamics by RNEA, the inverse of the joint-space mass matrix, forward
 * dynamics and the analytical gradient of forward dynamics. Robot models follow
 * Sec. III-B: bodies i = 0..n-1 with parent lambda_i < i, revolute joints with
 * motion subspace S_i = [a_i; 0], transforms iX_lambda_i = X_J(q_i) X_T,i and
 * spatial inertias I_i.
 *
 * Conventions for every compute call:
 *   - State arrays are caller-owned memory addressable by the device: device
 *     memory, or pinned host memory (cudaHostAlloc / cudaMallocHost, mapped in
 *     the unified address space), which the kernels then read and write
 *     directly over the CPU-GPU link (zero copy). They are knot-major and row-major:
 *     q[k*n + i] is joint i of knot point k. Matrices per knot point are
 *     row-major and contiguous: Minv[k*n*n + i*n + j], J[k*2n*n + i*2n + c].
 *     Joint order is the caller's numbering given to grid_create.
 *   - Pointers must be 4-byte aligned (8-byte for the _f64 calls); inputs and
 *     outputs must not overlap.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream). Nothing is allocated on these calls (except the
 *     staging of grid_grad_fd_host, which takes host buffers instead).
 *   - Arguments are checked synchronously; a launch failure is returned as
 *     GRID_E_CUDA. Errors raised inside a kernel surface at the caller's next
 *     synchronisation.
 *   - grid_last_error() returns a thread-local message for the last failure.
 *   - N = 0 is valid and does nothing.
 */
#ifndef GRID_H_
#define GRID_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct grid_model grid_model; /* opaque, library-owned */

typedef enum {
  GRID_OK = 0,
  GRID_E_ARG = 1,       /* null pointer, bad size, bad option */
  GRID_E_TOPOLOGY = 2,  /* parent[i] >= i or < -1, n out of range */
  GRID_E_ALIGN = 3,     /* misaligned pointer */
  GRID_E_CUDA = 4,      /* CUDA runtime error (message in grid_last_error) */
  GRID_E_NOMEM = 5,     /* device allocation failed (grid_create, grid_grad_fd_host staging) */
  GRID_E_TIMEOUT = 6,   /* bounded wait expired (serving) */
  GRID_E_NUMERIC = 7    /* non-physical model data (mass <= 0, axis not unit) */
} grid_status;

typedef enum {
  GRID_FP32 = 0,  /* all sweeps in FP32 */
  GRID_MIXED = 1, /* FP32, with the articulated-inertia pivots D_i = S_i^T I^A_i S_i
                     and their inverses (and the updates that divide by them) in FP64 */
  GRID_FP64 = 2   /* the whole path in FP64 (the _f64 calls) */
} grid_precision;

/* Largest supported number of moving joints (degrees of freedom). */
#define GRID_MAX_DOF 32

/* Joint types (Sec. IV-B lists revolute, prismatic and fixed joints). */
typedef enum {
  GRID_JOINT_REVOLUTE = 0,  /* rotation by q about the unit axis a: S = [a; 0] */
  GRID_JOINT_PRISMATIC = 1, /* translation of the child origin by q a: S = [0; a] */
  GRID_JOINT_FIXED = 2      /* no degree of freedom: merged into the parent at creation */
} grid_joint_type;

/*
 * grid_create -- build a device-resident robot model (Sec. III-B).
 *   n        number of revolute joints/bodies, 1 <= n <= GRID_MAX_DOF
 *   parent   [n] parent body of body i, -1 for the fixed base; parent[i] < i
 *   axis     [n][3] unit joint axis a_i in the joint frame (S_i = [a_i; 0])
 *   X_tree   [n][12] fixed transform X_T,i: E (3x3 row-major, maps parent
 *            coordinates to the joint's pre-rotation coordinates) then r (3,
 *            the joint origin expressed in the parent frame)
 *   inertia  [n][10] m, c[3] (centre of mass in the body frame), then the
 *            rotational inertia about the centre of mass: Ixx Iyy Izz Ixy Ixz Iyz
 *   gravity  [3] gravity vector in base coordinates, e.g. {0, 0, -9.81}
 *   prec     default precision of the float entry points (GRID_FP32 or
 *            GRID_MIXED); the _f64 entry points always run in FP64
 *   out      receives the model handle
 * Host pointers, read once. Allocates the device-resident model on the current
 * device (the device that later calls must use). Bodies are renumbered
 * internally in depth-first order; results are returned in the caller's order.
 * The model is immutable and may be used concurrently from several streams.
 */
grid_status grid_create(int n, const int* parent, const double* axis, const double* X_tree,
                        const double* inertia, const double* gravity, grid_precision prec,
                        grid_model** out);

/*
 * grid_create_ex -- grid_create with a joint type per body (Sec. IV-B: the
 * library supports revolute, prismatic and fixed joints).
 *   nb      number of bodies, 1 <= nb <= 256, at most GRID_MAX_DOF of them moving
 *   jtype   [nb] grid_joint_type per body, or NULL for all revolute
 *   parent, axis, X_tree, inertia, gravity, prec, out: as for grid_create, per
 *           body (axis is ignored for a fixed joint; a fixed body may have zero mass)
 * A prismatic joint translates the child origin by q a (X_J = X(1, q a),
 * S = [0; a]). A fixed body is merged into its nearest moving ancestor: its
 * spatial inertia is added to the ancestor's in the ancestor's frame and the
 * bodies hanging from it take the composed fixed transform (a fixed body on the
 * base contributes nothing). Every joint array of the compute calls (q, qd,
 * qdd, tau, and the rows and columns of M^-1 and the Jacobians) then holds the
 * moving joints only, in body order: grid_model_dof() of them.
 * Errors: GRID_E_ARG for a joint type outside 0..2, GRID_E_TOPOLOGY when no
 * joint moves or the limits are exceeded, GRID_E_NUMERIC for a non-unit axis of
 * a moving joint or a non-positive mass after merging.
 */
grid_status grid_create_ex(int nb, const int* parent, const int* jtype, const double* axis,
                           const double* X_tree, const double* inertia, const double* gravity,
                           grid_precision prec, grid_model** out);

/* grid_destroy -- free the model (synchronises the device first). NULL is a no-op. */
grid_status grid_destroy(grid_model* model);

/* grid_model_dof -- number of moving joints n of a model (0 for NULL). */
int grid_model_dof(const grid_model* model);

/*
 * grid_set_option -- tuning knobs (not needed for correctness).
 *   "lanes"       threads cooperating on one knot point: 0 = automatic, 1, 8, 16 or 32.
 *                 1: the float entry points (RNEA, M^-1, FD, gradients of ID and FD,
 *                 the vector-Jacobian product) of a serial chain of 2 to 8 revolute
 *                 bodies, and of a forest of such chains on the fixed base (each
 *                 chain in turn), run with one lane per knot point: the form that
 *                 batches of 32768 knot points or more take by default (not for
 *                 outputs in host memory); the gradient of FD also for chain
 *                 components of robots that run as parts. Elsewhere 1 acts as 0
 *   "precision"   GRID_FP32 or GRID_MIXED for the float entry points
 *   "ctas_per_sm" resident CTAs per SM the launcher sizes the grid for (0 = auto)
 *   "specialize"  1 (default): serial chains (parent[i] = i - 1) of 2 to 8 bodies,
 *                 and forests of 4 x 3, 2 x 6 or 4 x 4 equal chains on the base (in
 *                 depth-first order; with "lanes" 0),
 *                 run the gradient of FD (FP32 and FP64) in a kernel compiled for their
 *                 length (the chain topology of Sec. IV-C fixed at compile time); a
 *                 forest without fixed bodies runs as independent chains (its
 *                 chains do not interact through the fixed base);
 *                 2: as 1, and any other robot's gradient of FD runs in a kernel
 *                 compiled at run time (NVRTC, on the first call for each
 *                 precision and lane count) with its topology tables as constants;
 *                 GRID_E_CUDA if NVRTC or the driver library cannot be loaded;
 *                 0: always the kernel that reads the topology at run time
 *   "host_chunk"  knot points per chunk of grid_grad_fd_host (0 = automatic: about
 *                 32 MB of Jacobians per chunk)
 */
grid_status grid_set_option(grid_model* model, const char* key, int value);

/*
 * grid_rnea -- inverse dynamics tau = ID(q, qd, qdd) by the recursive
 * Newton-Euler algorithm (Sec. IV-B, first item; Featherstone ch. 5).
 *   q, qd [N][n]; qdd [N][n] or NULL for qdd = 0; tau [N][n] output.
 */
grid_status grid_rnea(const grid_model* model, int N, const float* q, const float* qd,
                      const float* qdd, float* tau, void* stream);

/*
 * grid_minv -- the inverse of the mass matrix M(q)^-1 computed directly,
 * without forming M, by the articulated-inertia recursion (Sec. IV-B, second
 * item; Carpentier 2018). Minv [N][n][n] output, full symmetric.
 */
grid_status grid_minv(const grid_model* model, int N, const float* q, float* Minv, void* stream);

/*
 * grid_fd -- forward dynamics qdd = M^-1 (tau - RNEA(q, qd, 0)) (Sec. IV-B,
 * third item). q, qd, tau [N][n]; qdd [N][n] output.
 */
grid_status grid_fd(const grid_model* model, int N, const float* q, const float* qd,
                    const float* tau, float* qdd, void* stream);

/*
 * grid_grad_fd -- analytical gradient of forward dynamics (Sec. IV-B, fifth
 * item): with qdd = FD(q, qd, tau), the analytical RNEA derivatives dID/dq and
 * dID/dqd (one column per joint, Alg. 1 / Alg. 2 and their backward pass) give
 *   [dqdd/dq | dqdd/dqd] = -M^-1 [dID/dq | dID/dqd].
 *   J   [N][n][2n] output; row i is qdd_i, columns 0..n-1 are d/dq_j,
 *       columns n..2n-1 are d/dqd_j.
 *   qdd [N][n] optional output (NULL to skip).
 * dqdd/dtau = M^-1 is available from grid_minv.
 */
grid_status grid_grad_fd(const grid_model* model, int N, const float* q, const float* qd,
                         const float* tau, float* J, float* qdd, void* stream);

/*
 * grid_grad_rnea -- analytical gradient of inverse dynamics (Sec. IV-B, fourth
 * item; Alg. 1 / Alg. 2 and their backward pass) at the given (q, qd, qdd):
 *   dID [N][n][2n] output; row i is tau_i, columns 0..n-1 are d/dq_j,
 *   columns n..2n-1 are d/dqd_j. qdd NULL means qdd = 0.
 */
grid_status grid_grad_rnea(const grid_model* model, int N, const float* q, const float* qd,
                           const float* qdd, float* dID, void* stream);

/*
 * grid_fd_vjp -- vector-Jacobian product through forward dynamics: for an
 * upstream gradient gbar = dL/dqdd at qdd = FD(q, qd, tau),
 *   dtau = M^-1 gbar,  dq = (dqdd/dq)^T gbar = -(dID/dq)^T M^-1 gbar,
 *   dqd = (dqdd/dqd)^T gbar = -(dID/dqd)^T M^-1 gbar
 * (Sec. IV-B, items 3 and 5, transposed). The RNEA derivatives are applied in
 * reverse mode (one adjoint sweep); no n x 2n Jacobian is formed and the
 * forward intermediates are recomputed from (q, qd, tau).
 *   q, qd, tau, gbar [N][n] inputs; dq, dqd, dtau [N][n] outputs.
 */
grid_status grid_fd_vjp(const grid_model* model, int N, const float* q, const float* qd,
                        const float* tau, const float* gbar, float* dq, float* dqd, float* dtau,
                        void* stream);

/* FP64 twins: same operations and layouts, the whole path in double. */
/*
 * grid_grad_fd_ex -- grid_grad_fd that also writes M^-1 = dqdd/dtau (Sec. IV-B,
 * fifth item), which the kernel forms on the way: Minv [N][n][n] full
 * symmetric, or NULL (then identical to grid_grad_fd).
 */
grid_status grid_grad_fd_ex(const grid_model* model, int N, const float* q, const float* qd,
                            const float* tau, float* J, float* qdd, float* Minv, void* stream);
grid_status grid_grad_fd_ex_f64(const grid_model* model, int N, const double* q, const double* qd,
                                const double* tau, double* J, double* qdd, double* Minv, void* stream);

/*
 * grid_grad_fd_host -- grid_grad_fd for data that lives in HOST memory: q, qd,
 * tau [N][n] in, J [N][n][2n] and, if qdd != NULL, qdd [N][n] out, in the layouts
 * above, all host pointers. The batch is cut into chunks of knot points
 * (option "host_chunk"; 0 = the default of about 32 MB of Jacobians per chunk)
 * that pass through three device staging slots owned by the model. The copy in
 * of chunk c+1, the kernel on chunk c and the copy out of chunk c-1 run at the
 * same time on three internal streams, so a call costs about the largest of the
 * two transfers and the kernel instead of their sum. Each array of each chunk
 * moves with one cudaMemcpyAsync.
 *   - Host buffers should be page-locked (cudaHostAlloc, cudaHostRegister);
 *     pageable memory gives the same results, with copies that do not overlap.
 *   - Ordering: the work starts after the work already queued on `stream`, and
 *     work queued on `stream` afterwards waits for its end. The call returns
 *     once everything is enqueued; the host buffers must stay valid and
 *     untouched until `stream` has reached that point (cudaStreamSynchronize).
 *   - Unlike the other compute calls this one allocates: the staging slots are
 *     allocated by the first call, replaced by larger ones when a later call
 *     needs bigger chunks (GRID_E_NOMEM if that fails), and freed by
 *     grid_destroy. Calls on one model are serialised (a host lock; events on
 *     the device), so a model may serve several threads and streams.
 *   - The results are those of grid_grad_fd on the same knot points, bit for
 *     bit where the kernel configuration does not depend on the number of knot
 *     points in a launch (serial chains and the compiled forests at 8 lanes);
 *     otherwise within rounding.
 */
grid_status grid_grad_fd_host(const grid_model* model, int N, const float* q, const float* qd,
                              const float* tau, float* J, float* qdd, void* stream);
grid_status grid_grad_fd_host_f64(const grid_model* model, int N, const double* q, const double* qd,
                                  const double* tau, double* J, double* qdd, void* stream);

/*
 * Trajectory-optimisation step (Sec. V-B: the all-GPU loop the library is built
 * for). Knot arrays are [B][H+1][n] (trajectory, knot point, joint): the
 * B (H+1) knot points of a batch are one contiguous set that grid_grad_fd_ex
 * differentiates in one call. Device (or pinned host) pointers; asynchronous
 * on `stream`; no allocation.
 *
 * grid_rollout -- semi-implicit Euler through forward dynamics:
 *   qdd_k = FD(q_k, qd_k, u_k), qd_{k+1} = qd_k + dt qdd_k, q_{k+1} = q_k + dt qd_{k+1}
 *   for k = 0 .. H-1 from q0, qd0 [B][n]. Without a policy (K = NULL) u_k = U_k;
 *   with one, u_k = U_k + alpha kff_k + K_k (x_k - xnom_k), x = (q, qd), with
 *   K [B][H+1][n][2n], kff [B][H+1][n] (from grid_riccati) and the nominal states
 *   Qnom, QDnom [B][H+1][n]. Outputs Q, QD [B][H+1][n] (knot 0 = q0, qd0) and,
 *   if Uout != NULL, the applied controls [B][H+1][n] (entry H set to 0).
 *   U's entry H is not read.
 *
 * grid_riccati -- the iLQR backward pass (DDP without second-order dynamics
 *   terms; Li and Todorov 2004, Tassa et al. 2012) for the tracking cost
 *     sum_{k<H} 1/2 (x_k - r_k)^T diag(wq) (x_k - r_k) + 1/2 u_k^T diag(wr) u_k
 *     + 1/2 (x_H - r_H)^T diag(wf) (x_H - r_H),   r = (Qref, QDref) [B][H+1][n]
 *   about the nominal trajectory (Q, QD, U). The step Jacobians come from J and
 *   Minv [B][H+1][n][2n], [B][H+1][n][n] (grid_grad_fd_ex at the nominal knots):
 *     A = [[1 + dt^2 Jq, dt (1 + dt Jv)], [dt Jq, 1 + dt Jv]],  B = [[dt^2 Minv], [dt Minv]].
 *   From V_x = diag(wf)(x_H - r_H), V_xx = diag(wf), for k = H-1 .. 0:
 *     Q_x = l_x + A^T V_x, Q_u = l_u + B^T V_x, Q_xx = l_xx + A^T V_xx A,
 *     Q_uu = l_uu + B^T V_xx B + mu 1, Q_ux = B^T V_xx A,
 *     K_k = -Q_uu^-1 Q_ux, k_k = -Q_uu^-1 Q_u,
 *     V_x = Q_x + K^T Q_uu k + K^T Q_u + Q_ux^T k,
 *     V_xx = sym(Q_xx + K^T Q_uu K + K^T Q_ux + Q_ux^T K).
 *   Outputs K [B][H+1][n][2n] and kff [B][H+1][n] (entry H set to 0) and
 *   dV [B][2] = (sum k^T Q_u, sum 1/2 k^T Q_uu k): the predicted cost change of a
 *   step alpha is alpha dV[0] + alpha^2 dV[1]. A trajectory whose Q_uu is not
 *   positive definite at some step gets dV = NaN (raise mu). Weights wq, wf [2n]
 *   and wr [n] in device memory. Requires n <= 16 (GRID_E_ARG otherwise).
 */
grid_status grid_rollout(const grid_model* model, int B, int H, float dt, const float* q0,
                         const float* qd0, const float* U, const float* K, const float* kff,
                         const float* Qnom, const float* QDnom, float alpha, float* Q, float* QD,
                         float* Uout, void* stream);
grid_status grid_rollout_f64(const grid_model* model, int B, int H, double dt, const double* q0,
                             const double* qd0, const double* U, const double* K, const double* kff,
                             const double* Qnom, const double* QDnom, double alpha, double* Q,
                             double* QD, double* Uout, void* stream);
grid_status grid_riccati(const grid_model* model, int B, int H, float dt, const float* Q,
                         const float* QD, const float* U, const float* J, const float* Minv,
                         const float* Qref, const float* QDref, const float* wq, const float* wr,
                         const float* wf, float mu, float* K, float* kff, float* dV, void* stream);
grid_status grid_riccati_f64(const grid_model* model, int B, int H, double dt, const double* Q,
                             const double* QD, const double* U, const double* J, const double* Minv,
                             const double* Qref, const double* QDref, const double* wq,
                             const double* wr, const double* wf, double mu, double* K, double* kff,
                             double* dV, void* stream);

grid_status grid_rnea_f64(const grid_model* model, int N, const double* q, const double* qd,
                          const double* qdd, double* tau, void* stream);
grid_status grid_minv_f64(const grid_model* model, int N, const double* q, double* Minv, void* stream);
grid_status grid_fd_f64(const grid_model* model, int N, const double* q, const double* qd,
                        const double* tau, double* qdd, void* stream);
grid_status grid_grad_fd_f64(const grid_model* model, int N, const double* q, const double* qd,
                             const double* tau, double* J, double* qdd, void* stream);
grid_status grid_grad_rnea_f64(const grid_model* model, int N, const double* q, const double* qd,
                               const double* qdd, double* dID, void* stream);
grid_status grid_fd_vjp_f64(const grid_model* model, int N, const double* q, const double* qd,
                            const double* tau, const double* gbar, double* dq, double* dqd,
                            double* dtau, void* stream);

/*
 * Serving: a persistent kernel computes grid_grad_fd for a stream of requests
 * (mixed robots and horizons) with continuous batching. Requests are published
 * into a ring of `ring_slots` slots in mapped pinned host memory; their states
 * and Jacobians live in a pinned I/O arena of `arena_bytes` that the GPU reads
 * and writes directly. A submission is admitted when its ring slot is free and
 * its I/O fits in the arena; otherwise it returns GRID_E_NOMEM and the caller
 * retries after collecting results. Tiles of 2 knot points from all published
 * requests are claimed by warps in publication order, so requests that arrive
 * while others run start at once and overlap on the device. Every wait in the
 * kernel is bounded: with no new work for the idle timeout (default 2 s) the
 * kernel ends with GRID_E_TIMEOUT. All models must be FP32 models of the
 * current device (GRID_E_ARG for a GRID_MIXED model: the serving kernel has no
 * FP64 pivots); the server runs in FP32 with 16 lanes per knot point.
 */
typedef struct grid_server grid_server;

/* grid_server_create -- allocate the ring, control block and arena (host). */
grid_status grid_server_create(const grid_model* const* models, int nmodels, int ring_slots,
                               size_t arena_bytes, grid_server** out);
/* grid_server_set_idle_timeout -- idle limit of the persistent kernel (before start). */
grid_status grid_server_set_idle_timeout(grid_server* server, double seconds);
/* grid_server_start -- launch the persistent kernel on `stream` (asynchronous; NULL = a
 * non-blocking stream of the server's own, so that it neither waits for nor holds up
 * work on the legacy default stream). */
grid_status grid_server_start(grid_server* server, void* stream);
/*
 * grid_server_submit -- copy one request's host states (q, qd, tau: [H][n],
 * n of model `model`) into the arena and publish it; *request_id receives its
 * id. GRID_E_NOMEM: no free slot or arena space right now.
 */
grid_status grid_server_submit(grid_server* server, int model, int H, const float* q,
                               const float* qd, const float* tau, long long* request_id);
/*
 * grid_server_result -- wait up to wait_us microseconds (0 = poll once) for a
 * request; on success copy its Jacobians [H][n][2n] to host J (NULL to skip)
 * and release its slot and arena space. GRID_E_TIMEOUT if not done yet or the
 * kernel has stopped.
 */
grid_status grid_server_result(grid_server* server, long long request_id, float* J, int wait_us);
/* grid_server_stop -- ask the kernel to exit, wait for it, return its status. */
grid_status grid_server_stop(grid_server* server);
/* grid_server_kernel_status -- GRID_OK while healthy, GRID_E_TIMEOUT after an idle exit. */
int grid_server_kernel_status(const grid_server* server);
/* grid_server_destroy -- stop if running and free everything. */
grid_status grid_server_destroy(grid_server* server);
/*
 * grid_server_bench -- open-loop Poisson load for `seconds` at `rate_hz`:
 * robot uniform over the server's models, horizon uniform over horizons[nh],
 * states sliced from pools[model] ([3][pool_knots][n]: q, qd, tau). Latency
 * runs from each scheduled arrival to the host seeing its done flag.
 * stats[9]: completed, knot points, wall s, p50 ms, p99 ms, p50 ms (H = 128),
 * p99 ms (H = 128), max ms, refused submissions.
 */
grid_status grid_server_bench(grid_server* server, double rate_hz, double seconds,
                              unsigned long long seed, const int* horizons, int nh,
                              const float* const* pools, int pool_knots, double* stats);

/*
 * grid_serve_batch_static -- gradient of FD for a fixed list of requests of
 * mixed robots and horizons, without allocating anything. (The paper has no
 * counterpart; this serves callers that may not allocate device memory once
 * running, such as a real-time control loop, where cudaMalloc can synchronise
 * the device and take unbounded time, or a host application that owns all
 * device memory and only lends the library its buffers.)
 *   models[nmodels]     FP32 models of the current device (GRID_E_ARG for a
 *                       GRID_MIXED model: the serving kernel has no FP64 pivots)
 *   req_model, req_H    host arrays [nreq]: model index and knot points
 *   q, qd, tau          host arrays [nreq] of DEVICE pointers, each [H][n]
 *   J                   host array [nreq] of DEVICE pointers, each [H][n][2n]
 * Runs the serving kernel in one-shot form on `stream`. Its scratch (request
 * descriptors, control block, counters) is a fixed array of about 18.5 KB that
 * the library holds on every device it is loaded on until the process exits;
 * 1 <= nreq <= 256 per call, larger lists are refused with GRID_E_ARG. The
 * first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture. The request list goes to the device by value as the argument of a
 * small set-up kernel on `stream`, which also clears the array's counters; the
 * host arrays may be reused as soon as the call returns. Calls share the array
 * and overwrite its contents, so calls that overlap on the GPU (different
 * streams, or another call before this one's kernel has finished) race;
 * serialise them. Every request is published before the launch, so the
 * kernel's waits and its request search always succeed; the call reports
 * argument and launch errors, and a fault inside a kernel surfaces at the
 * caller's next synchronisation, as for every compute call. (The serving
 * kernel's own status word, which its bounded waits set when they give up,
 * sits in the fixed array and is not read back by this call: with every
 * request published before the launch, those waits do not give up.)
 */
grid_status grid_serve_batch_static(const grid_model* const* models, int nmodels, int nreq,
                                    const int* req_model, const int* req_H, const float* const* q,
                                    const float* const* qd, const float* const* tau, float* const* J,
                                    void* stream);

/*
 * grid_peak_loop -- arithmetic-throughput loop, the denominator of a roofline
 * fraction (a measurement utility; not part of the paper's method). Launches
 * `blocks` x `threads` threads on `stream`; each runs `iters` iterations of 8
 * independent multiply-add chains held in registers, then writes one value to
 * out[block * threads + thread]:
 *   kind 0  FP32 fma          (out: float [blocks * threads])
 *   kind 1  paired FP32 fma   (two independent multiply-adds per instruction; out: float)
 *   kind 2  FP64 fma          (out: double [blocks * threads])
 * *flops receives the floating-point operations of the launch (2 per
 * multiply-add); divide by the launch's duration (CUDA events on `stream`).
 * threads: a multiple of 32 up to 1024. GRID_E_ARG for bad arguments.
 */
grid_status grid_peak_loop(int kind, int blocks, int threads, int iters, void* out, double* flops,
                           void* stream);

/* grid_last_error -- thread-local description of the last failure ("" if none). */
const char* grid_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GRID_H_ */
