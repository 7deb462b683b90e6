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
 *   - State arrays are caller-owned DEVICE memory, knot-major and row-major:
 *     q[k*n + i] is joint i of knot point k. Matrices per knot point are
 *     row-major and contiguous: Minv[k*n*n + i*n + j], J[k*2n*n + i*2n + c].
 *     Joint order is the caller's numbering given to grid_create.
 *   - Pointers must be 4-byte aligned (8-byte for the _f64 calls); inputs and
 *     outputs must not overlap.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream). Nothing is allocated on these calls.
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
  GRID_E_NOMEM = 5,     /* device allocation failed in grid_create */
  GRID_E_TIMEOUT = 6,   /* bounded wait expired (serving) */
  GRID_E_NUMERIC = 7    /* non-physical model data (mass <= 0, axis not unit) */
} grid_status;

typedef enum {
  GRID_FP32 = 0,  /* all sweeps in FP32 */
  GRID_MIXED = 1, /* FP32, with the articulated-inertia pivots D_i = S_i^T I^A_i S_i
                     and their inverses (and the updates that divide by them) in FP64 */
  GRID_FP64 = 2   /* the whole path in FP64 (the _f64 calls) */
} grid_precision;

/* Largest supported number of joints. */
#define GRID_MAX_DOF 32

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

/* grid_destroy -- free the model (synchronises the device first). NULL is a no-op. */
grid_status grid_destroy(grid_model* model);

/* grid_model_dof -- number of joints n of a model (0 for NULL). */
int grid_model_dof(const grid_model* model);

/*
 * grid_set_option -- tuning knobs (not needed for correctness).
 *   "lanes"       threads cooperating on one knot point: 0 = automatic, 8, 16 or 32
 *   "precision"   GRID_FP32 or GRID_MIXED for the float entry points
 *   "ctas_per_sm" resident CTAs per SM the launcher sizes the grid for (0 = auto)
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
grid_status grid_rnea_f64(const grid_model* model, int N, const double* q, const double* qd,
                          const double* qdd, double* tau, void* stream);
grid_status grid_minv_f64(const grid_model* model, int N, const double* q, double* Minv, void* stream);
grid_status grid_fd_f64(const grid_model* model, int N, const double* q, const double* qd,
                        const double* tau, double* qdd, void* stream);
grid_status grid_grad_fd_f64(const grid_model* model, int N, const double* q, const double* qd,
                             const double* tau, double* J, double* qdd, void* stream);
grid_status grid_fd_vjp_f64(const grid_model* model, int N, const double* q, const double* qd,
                            const double* tau, const double* gbar, double* dq, double* dqd,
                            double* dtau, void* stream);

/* grid_last_error -- thread-local description of the last failure ("" if none). */
const char* grid_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GRID_H_ */
