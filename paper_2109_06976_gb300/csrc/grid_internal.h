// Internal model representation shared by the host builder and the kernels.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "../../include/grid.h"


// Small type traits (these headers are also compiled at run time by NVRTC,
// which has no standard library).
template <class A, class B> struct grid_same { static constexpr bool value = false; };
template <class A> struct grid_same<A, A> { static constexpr bool value = true; };
template <bool C, class A, class B> struct grid_cond { using type = A; };
template <class A, class B> struct grid_cond<false, A, B> { using type = B; };

#ifdef __CUDACC__
#define GRID_HD __host__ __device__
#else
#define GRID_HD
#endif

// Kernel modes (one kernel template serves every entry point).
enum { MODE_RNEA = 0, MODE_MINV = 1, MODE_FD = 2, MODE_GRAD = 3, MODE_VJP = 4, MODE_GRAD_ID = 5 };

#define GRID_SCHED_MAX 4096    // step descriptors for all lane counts together
#define GRID_NUM_LANE_CFG 3    // lanes per knot point: 8, 16, 32

// Column-phase step descriptor (one uint32 per lane per step).
//   bits 0-4   body k (internal numbering)
//   bits 5-10  output column (u * n + j)
//   bit 11     RESET: first step of a path, parent derivatives are zero
//   bit 12     ROOT: body k is the column's joint j (case terms of Alg. 1)
//   bit 13     OWNED: first path through k; its force derivative is counted
//   bit 14     FLUSH: last step of a path; accumulators are written out
//   bit 15     UQ: column is d/dq_j (else d/dqd_j)
//   bit 16     VALID: real work (padding steps have it clear)
//   bits 17-21 depth of body k
//   bits 22-31 first subspace row of body k (skoff[k])
#define STEP_BODY(s) ((int)((s) & 31u))
#define STEP_COL(s) ((int)(((s) >> 5) & 63u))
#define STEP_RESET (1u << 11)
#define STEP_ROOT (1u << 12)
#define STEP_OWNED (1u << 13)
#define STEP_FLUSH (1u << 14)
#define STEP_UQ (1u << 15)
#define STEP_VALID (1u << 16)
#define STEP_DEPTH(s) ((int)(((s) >> 17) & 31u))
#define STEP_SKOFF(s) ((int)((s) >> 22))

// Offsets (in scalars) of the per-knot shared-memory workspace.
struct KnotLayout {
  int Q, QD, TAU, QDD, CB;      // staged q, qd, tau (or qdd input), qdd, bias force / tau out
  int X;                        // per body E(9) r(3)
  int VG, BPH;                  // per body 12: v | gamma = I v, and beta = (X a_parent) x S | phi = S x* F
  int MINV, MS;                 // n x n with row stride MS (a multiple of 4)
  int SK;                       // per body (depth + 1) rows of 8: ancestor subspaces s_m^(k)
  int UNION;                    // start of the phase-dependent area
  // M^-1 temporaries, relative to UNION
  int UB, DINV, CT, BIA, BP;    // U_i (8n), D_i^-1 (n, doubles in mixed mode), congruence exchange (2 x 6 x 8),
                                // branch-body I^A contributions (36 each), branch-body P columns (6n each)
  // RNEA temporaries, relative to UNION
  int A, F, FSL, GR;            // per body 8: acceleration, force (own, then accumulated in place);
                                // FSL: force contributions to branch bodies (8 each);
                                // GR: gravity rows g^(k) = kX_0 a_0 (8 per body), clear of the M^-1 area
  // derivative-column temporaries and output staging, relative to UNION
  int DC, JS;                   // dc [n][2n]; output staging in caller order (not in the gradient layout)
  // vector-Jacobian product (VJP layout only), relative to UNION, after the RNEA temporaries
  int GB, LAM, PSI, AB, VB, SA, SV, DQ, DQD;  // gbar (caller order), lambda, psi, adjoint seeds (8n each),
                                              // branch slots (8 each), dL/dq, dL/dqd (internal order)
  int stride;                   // scalars per knot
};

GRID_HD constexpr int grid_round_up(int x, int m) { return (x + m - 1) / m * m; }
GRID_HD constexpr int grid_imax(int a, int b) { return a > b ? a : b; }
GRID_HD constexpr int grid_take(int& off, int count) {
  const int o = off;
  off += grid_round_up(count, 4);
  return o;
}

// Workspace layout of one knot point for n bodies, nsk subspace rows and
// nbranch branch bodies. ssize is the scalar size in bytes; kind 0 is the
// gradient-of-FD kernel (J stored directly), 1 the kernels that stage their
// outputs, 2 the vector-Jacobian product. Evaluated on the host for every model
// and at compile time for the topology-specialised kernels.
GRID_HD constexpr KnotLayout make_layout(int n, int nsk, int nbranch, int ssize, int kind) {
  KnotLayout L{};
  int off = 0;
  L.Q = grid_take(off, n); L.QD = grid_take(off, n); L.TAU = grid_take(off, n);
  L.QDD = grid_take(off, n); L.CB = grid_take(off, n);
  L.X = grid_take(off, 12 * n);
  L.VG = grid_take(off, 12 * n); L.BPH = grid_take(off, 12 * n);
  L.MS = grid_round_up(n, 4);
  L.MINV = grid_take(off, n * L.MS);
  L.SK = grid_take(off, 8 * nsk);
  L.UNION = off;
  int b = 0;                                          // M^-1 temporaries
  L.UB = grid_take(b, 8 * n);
  L.DINV = grid_take(b, ssize == 4 ? 2 * n : n);      // doubles (mixed mode stores them in pairs of floats)
  L.CT = grid_take(b, 48);                            // one 6 x 8 buffer
  L.BIA = grid_take(b, 36 * nbranch);
  L.BP = grid_take(b, 6 * n * nbranch);
  int r = 0;                                          // RNEA temporaries
  L.A = grid_take(r, 8 * n); L.F = grid_take(r, 8 * n); L.FSL = grid_take(r, 8 * nbranch);
  r = grid_imax(r, b);                                // gravity rows are written while M^-1 runs
  L.GR = grid_take(r, 8 * n);
  if (kind == 2) {
    L.GB = grid_take(r, n); L.LAM = grid_take(r, n); L.PSI = grid_take(r, 8 * n);
    L.AB = grid_take(r, 8 * n); L.VB = grid_take(r, 8 * n);
    L.SA = grid_take(r, 8 * nbranch); L.SV = grid_take(r, 8 * nbranch);
    L.DQ = grid_take(r, n); L.DQD = grid_take(r, n);
  }
  const int c = 2 * n * n;                            // dc
  L.DC = 0;
  int u = grid_imax(b, grid_imax(r, c));
  if (kind == 1) { L.JS = u; u += grid_round_up(2 * n * n, 4); }
  if (kind == 2) { L.JS = u; u += grid_round_up(3 * n, 4); }
  off += grid_round_up(u, 4);
  // Knot stride: 16 bytes more than a multiple of 128 bytes (the 32 banks), so
  // that the knot points of a warp touching the same field start in different
  // bank quads. Measured on the 7-DoF step against 48, 64 and 80 bytes more:
  // 1654 against 1678 to 1863 shared-memory wavefronts per tile of 4 knot
  // points, the fewest bank conflicts and the shortest time.
  const int rb = 16 / ssize, qq = 128 / ssize;        // in scalars
  L.stride = (off + qq - rb - 1) / qq * qq + rb;
  return L;
}

GRID_HD constexpr int layout_kind(int mode) { return mode == MODE_GRAD ? 0 : (mode == MODE_VJP ? 2 : 1); }

#define GRID_MAX_BODIES 256       // bodies before fixed joints are merged

template <class S>
struct ModelDev {
  int n, maxd, nsk, ncomp, nbranch;
  int any_prism;                 // some joint is prismatic
  int steps[GRID_NUM_LANE_CFG];      // steps per lane for 8, 16, 32 lanes
  int sched_off[GRID_NUM_LANE_CFG];  // offsets into sched
  KnotLayout L;                  // workspace of the gradient-of-FD kernel (J is stored directly)
  KnotLayout LS;                 // workspace of the RNEA / M^-1 / FD / gradient-of-ID kernels (staged outputs)
  KnotLayout LV;                 // workspace of the vector-Jacobian-product kernel
  int parent[GRID_MAX_DOF];
  int depth[GRID_MAX_DOF];
  int sub_end[GRID_MAX_DOF];
  int comp_lo[GRID_MAX_DOF];
  int comp_hi[GRID_MAX_DOF];
  int perm[GRID_MAX_DOF];        // internal body -> caller index
  int skoff[GRID_MAX_DOF];       // first subspace row of body k
  int branch[GRID_MAX_DOF];      // slot of a body with >= 2 children, else -1
  int et_ident[GRID_MAX_DOF];
  int jt[GRID_MAX_DOF];          // GRID_JOINT_REVOLUTE or GRID_JOINT_PRISMATIC
  // Placement in the caller's arrays. A whole robot has ld = n, gslot and gidx
  // (below, read from device memory) the identity and perm. A part (one base
  // component of a robot, run as a problem of its own) has ld = the robot's
  // joints per knot point: its caller slot s is the robot's joint gslot[s], its
  // internal body k the robot's joint gidx[k] = gslot[perm[k]], and gmask has a
  // bit for each of its joints.
  int ld;
  unsigned gmask;
  alignas(16) S axis[GRID_MAX_DOF][4];   // unit axis, padded
  S ET[GRID_MAX_DOF][9];
  S rT[GRID_MAX_DOF][3];
  alignas(16) S inert[GRID_MAX_DOF][12]; // m, h = m c (3), Ibar about the origin: xx yy zz xy xz yz, pad
  alignas(16) S a0[8];                   // base acceleration -g, padded
  // -- not staged into shared memory:
  alignas(16) S Icol[GRID_MAX_DOF][6][8];// columns of the 6x6 spatial inertia, padded
  int gslot[GRID_MAX_DOF];       // placement tables of a part (see ld)
  int gidx[GRID_MAX_DOF];
  uint32_t sched[GRID_SCHED_MAX];
};

template <int MODE, class S>
GRID_HD inline const KnotLayout& layout_of(const ModelDev<S>& m) {
  return MODE == MODE_VJP ? m.LV : (MODE == MODE_GRAD ? m.L : m.LS);
}

// Bytes of ModelDev that every CTA copies into shared memory (everything up to
// the inertia column table, which is read from device memory, and the
// schedules, whose lane-count slice is copied separately).
template <class S>
GRID_HD constexpr int model_head_bytes() {
#ifdef __CUDACC_RTC__   // run-time compilation: the library passes the offsets it was built with
  return sizeof(S) == 4 ? GRID_RTC_HEAD_F : GRID_RTC_HEAD_D;
#else
  return (int)offsetof(ModelDev<S>, Icol);
#endif
}

struct grid_model {
  int n;
  int device;
  grid_precision prec;
  int lanes_opt;
  int ctas_opt;
  int chain;                     // parent[i] = i - 1 for every body (a serial chain)
  int forest_k, forest_l;        // K >= 2 equal chains of L revolute bodies on the base, else 0
  int branches;                  // K when the forest also has one model per chain (below), else 0
  ModelDev<float>* br_dev_f;     // the K chain models: device arrays and host mirrors
  ModelDev<double>* br_dev_d;
  ModelDev<float>* br_host_f;
  ModelDev<double>* br_host_d;
  int nparts;                    // > 0: the gradient of FD runs per base component
  struct grid_part* parts;       // [nparts] (grid_capi.cu), else nullptr
  struct grid_part_exec* pexec;  // streams and events that run the parts at once (grid_capi.cu)
  struct grid_gen_cache* gen;    // kernels compiled at run time for this model (grid_nvrtc.cpp)
  struct grid_host_pipe* pipe;   // staging and streams of grid_grad_fd_host (grid_capi.cu)
  int host_chunk_opt;            // knot points per chunk of grid_grad_fd_host (0 = automatic)
  int specialize_opt;            // use the topology-specialised kernels where one exists (default 1)
  ModelDev<float>* dev_f;        // device copies
  ModelDev<double>* dev_d;
  ModelDev<float>* host_f;       // host mirrors (for launch decisions)
  ModelDev<double>* host_d;
};

// One base component of a robot whose components differ: its own model
// (placed in the robot's arrays, see ModelDev::ld) and whether it is a serial
// chain of revolute joints in caller order.
struct grid_part {
  int n;
  int chain;
  ModelDev<float>* dev_f;
  ModelDev<double>* dev_d;
  ModelDev<float>* host_f;
  ModelDev<double>* host_d;
};

// Run-time specialisation (grid_nvrtc.cpp)
void grid_gen_cache_free(struct grid_gen_cache* c);

// Host helpers (grid_host.cpp)
void grid_set_error(const char* fmt, ...);
grid_status grid_build_model(int nb, const int* parent, const int* jtype, const double* axis,
                             const double* X_tree, const double* inertia, const double* gravity,
                             ModelDev<float>* mf, ModelDev<double>* md);
