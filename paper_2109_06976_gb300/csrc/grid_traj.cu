// Trajectory-optimisation step on the device: a rollout through forward
// dynamics (optionally under a feedback policy) and the iLQR backward pass,
// whose step Jacobians come from the analytical gradient of FD and M^-1
// (grid_grad_fd_ex). Sec. V-B names the all-GPU trajectory-optimisation loop
// as the use GRiD targets; the recursions are the textbook forms (Li and
// Todorov 2004; Tassa, Erez and Todorov 2012).
//
// Knot arrays are [B][H+1][n]: trajectory b, knot point k, joint i, so the
// B (H+1) knot points of a batch are one contiguous set for grid_grad_fd_ex.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <initializer_list>
#include <type_traits>

#include "grid_launch.cuh"

// iLQR backward pass, compiled per state size (grid_riccati.cu)
template <class S>
grid_status launch_riccati(const grid_model* m, int B, int H, S dt, const S* Q, const S* QD, const S* U,
                           const S* J, const S* Minv, const S* Qr, const S* QDr, const S* wq, const S* wr,
                           const S* wf, S mu, S* K, S* kff, S* dV, cudaStream_t st);

namespace {

// ---------------------------------------------------------------- rollout
// qdd_k = FD(q_k, qd_k, u_k), qd_{k+1} = qd_k + dt qdd_k, q_{k+1} = q_k + dt qd_{k+1};
// with a policy u_k = U_k + alpha kff_k + K_k (x_k - xnom_k). One knot slot of
// a warp per trajectory (T lanes), the H steps in sequence; the state stays in
// the slot's workspace between steps. CHAIN_N > 0: a serial chain of that many
// bodies, whose topology the phases then take at compile time.
template <class S, int T, int CPL, bool MIXED, int CHAIN_N = 0>
__global__ void __launch_bounds__(128) rollout_kernel(
    const ModelDev<S>* __restrict__ gm, int B, int H, S dt, const S* __restrict__ q0,
    const S* __restrict__ qd0, const S* __restrict__ U, const S* __restrict__ K, const S* __restrict__ kff,
    const S* __restrict__ Qn, const S* __restrict__ QDn, S alpha, S* __restrict__ Q, S* __restrict__ QD,
    S* __restrict__ Uout) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int head = align16(model_head_bytes<S>());
  {
    const int4* src = reinterpret_cast<const int4*>(gm);
    int4* dst = reinterpret_cast<int4*>(smem);
    for (int i = threadIdx.x; i < head / 16; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  using P = typename std::conditional<MIXED, double, S>::type;
  using Tp = topo_for<S, MODE_FD, CHAIN_N>;
  const ModelDev<S>& M = *reinterpret_cast<const ModelDev<S>*>(smem);
  const Tp tp(M);
  const KnotLayout& L = tp.layout();
  const int n = tp.n();
  constexpr int G = 32 / T;
  const int lane32 = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int g = lane32 / T, l = lane32 % T;
  S* W = reinterpret_cast<S*>(smem + head) + (warp * G + g) * L.stride;
  const Ctx<S, Tp> c{M, gm, tp, W, l, lane32};
  const size_t knots = (size_t)H + 1;
  const int ntiles = (B + G - 1) / G;
  for (int tile = blockIdx.x * wpb + warp; tile < ntiles; tile += gridDim.x * wpb) {
    const int b = tile * G + g;
    const bool ok = b < B;                     // padding slots compute on zeros and store nothing
    const size_t k0 = (size_t)(ok ? b : 0) * knots;
    for (int i = l; i < n; i += T) {
      const S qv = ok ? q0[(size_t)b * n + i] : S(0);
      const S qdv = ok ? qd0[(size_t)b * n + i] : S(0);
      W[L.Q + i] = qv;
      W[L.QD + i] = qdv;
      if (ok) { Q[k0 * n + i] = qv; QD[k0 * n + i] = qdv; }
    }
    SYNC();
    for (int k = 0; k < H; ++k) {
      const size_t kb = k0 + k;
      for (int i = l; i < n; i += T) {       // control of step k (caller order)
        S u = ok ? U[kb * n + i] : S(0);
        if (K && ok) {
          const S* Kr = K + (kb * n + i) * 2 * n;
          S acc = alpha * kff[kb * n + i];
          for (int j = 0; j < n; ++j)
            acc += Kr[j] * (W[L.Q + j] - Qn[kb * n + j]) + Kr[n + j] * (W[L.QD + j] - QDn[kb * n + j]);
          u += acc;
        }
        W[L.TAU + i] = u;
        if (ok && Uout) Uout[kb * n + i] = u;
      }
      SYNC();
      ph_transforms<S, T>(c);
      ph_minv<S, P, T, CPL, true>(c);
      ph_rnea_bodies<S, T>(c, -1);
      ph_joint_forces<S, T>(c, L.UNION + L.F, L.CB);
      ph_fd<S, T>(c);
      for (int i = l; i < n; i += T) {       // semi-implicit Euler; qdd is in internal order
        const int ci = tp.perm(i);
        const S qd1 = W[L.QD + ci] + dt * W[L.QDD + i];
        const S q1 = W[L.Q + ci] + dt * qd1;
        W[L.QD + ci] = qd1;
        W[L.Q + ci] = q1;
        if (ok) { Q[(kb + 1) * n + ci] = q1; QD[(kb + 1) * n + ci] = qd1; }
      }
      SYNC();
    }
    if (ok && Uout)
      for (int i = l; i < n; i += T) Uout[(k0 + H) * n + i] = S(0);
    SYNC();
  }
}

// Warps per CTA with the most resident warps (same rule as the dynamics kernels).
template <class Kern>
bool pick_launch(Kern kern, int dev_optin, size_t fixed, size_t per_warp, int& warps, int& per_sm) {
  int best = 0;
  warps = per_sm = 0;
  for (int w = 4; w >= 1; --w) {
    const size_t sm = fixed + w * per_warp;
    if (sm > (size_t)dev_optin) continue;
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, 32 * w, sm);
    if (blocks * w > best) { best = blocks * w; warps = w; per_sm = blocks; }
  }
  return warps > 0;
}

template <class S, int T, int CPL, bool MIXED, int CHAIN_N = 0>
grid_status launch_rollout(const grid_model* m, const ModelDev<S>* hm, const ModelDev<S>* dm, int B, int H, S dt,
                           const S* q0, const S* qd0, const S* U, const S* K, const S* kff, const S* Qn,
                           const S* QDn, S alpha, S* Q, S* QD, S* Uout, cudaStream_t st) {
  auto kern = rollout_kernel<S, T, CPL, MIXED, CHAIN_N>;
  if constexpr (CHAIN_N > 0) {               // the compile-time layout must be the one the host built
    if (hm->n != CHAIN_N || ChainTopo<S, MODE_FD, CHAIN_N>::layout().stride != hm->LS.stride) {
      grid_set_error("rollout chain kernel for %d bodies does not match the model", CHAIN_N);
      return GRID_E_TOPOLOGY;
    }
  }
  const DevInfo di = dev_info(m->device);
  static std::atomic<int> opted{0};
  if (!opted.load()) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, di.smem_optin) != cudaSuccess) {
      grid_set_error("cudaFuncSetAttribute failed");
      return GRID_E_CUDA;
    }
    opted.store(1);
  }
  constexpr int G = 32 / T;
  const size_t fixed = align16(model_head_bytes<S>());
  const size_t per_warp = (size_t)G * hm->LS.stride * sizeof(S);
  int warps, per_sm;
  if (!pick_launch(kern, di.smem_optin, fixed, per_warp, warps, per_sm)) {
    grid_set_error("rollout workspace needs %zu B of shared memory per warp; use more lanes", fixed + per_warp);
    return GRID_E_ARG;
  }
  const long tiles = (B + G - 1) / G;
  const int grid = (int)std::min<long>((tiles + warps - 1) / warps, (long)di.nsm * per_sm);
  kern<<<grid, 32 * warps, fixed + warps * per_warp, st>>>(dm, B, H, dt, q0, qd0, U, K, kff, Qn, QDn, alpha, Q, QD,
                                                           Uout);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    grid_set_error("rollout launch: %s", cudaGetErrorString(err));
    return GRID_E_CUDA;
  }
  return GRID_OK;
}

template <class S, bool MIXED>
grid_status rollout_dispatch(const grid_model* m, int B, int H, S dt, const S* q0, const S* qd0, const S* U,
                             const S* K, const S* kff, const S* Qn, const S* QDn, S alpha, S* Q, S* QD, S* Uout,
                             cudaStream_t st) {
  const ModelDev<S>* hm;
  const ModelDev<S>* dm;
  if constexpr (std::is_same<S, float>::value) { hm = m->host_f; dm = m->dev_f; }
  else { hm = m->host_d; dm = m->dev_d; }
  const int n = hm->n;
  int T = m->lanes_opt;
  if (T == 0 || T == 1) T = n <= 12 ? 8 : 16;
  const int cpl = (n + T - 1) / T;
  // serial chains of 2 .. 8 bodies: the chain topology at compile time (8 lanes)
  if (!MIXED && m->chain && m->specialize_opt && T == 8 && n >= 2 && n <= kChainMaxN) {
    switch (n) {
#define GRID_RLC(NB) \
      case NB: return launch_rollout<S, 8, 1, MIXED, NB>(m, hm, dm, B, H, dt, q0, qd0, U, K, kff, Qn, QDn, alpha, \
                                                          Q, QD, Uout, st);
      GRID_RLC(2) GRID_RLC(3) GRID_RLC(4) GRID_RLC(5) GRID_RLC(6) GRID_RLC(7) GRID_RLC(8)
#undef GRID_RLC
      default: break;
    }
  }
#define GRID_RL(TT, CC) return launch_rollout<S, TT, CC, MIXED>(m, hm, dm, B, H, dt, q0, qd0, U, K, kff, Qn, QDn, \
                                                                  alpha, Q, QD, Uout, st)
  if (T == 8) { if (cpl <= 1) GRID_RL(8, 1); if (cpl <= 2) GRID_RL(8, 2); GRID_RL(8, 4); }
  if (T == 16) { if (cpl <= 1) GRID_RL(16, 1); GRID_RL(16, 2); }
  if (T == 32) GRID_RL(32, 1);
#undef GRID_RL
  grid_set_error("lanes option %d not in {0, 8, 16, 32}", T);
  return GRID_E_ARG;
}

template <class S>
grid_status check_traj(const grid_model* m, int B, int H, std::initializer_list<const void*> must,
                       std::initializer_list<const void*> may) {
  if (!m) { grid_set_error("null model"); return GRID_E_ARG; }
  if (B < 0 || H < 1) { grid_set_error("B = %d, H = %d (need B >= 0, H >= 1)", B, H); return GRID_E_ARG; }
  for (const void* p : must) {
    if (!p && B > 0) { grid_set_error("null trajectory pointer"); return GRID_E_ARG; }
    if (((uintptr_t)p) % sizeof(S)) { grid_set_error("pointer not %zu-byte aligned", sizeof(S)); return GRID_E_ALIGN; }
  }
  for (const void* p : may)
    if (((uintptr_t)p) % sizeof(S)) { grid_set_error("pointer not %zu-byte aligned", sizeof(S)); return GRID_E_ALIGN; }
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != m->device) {
    grid_set_error("current device %d differs from the model's device %d", dev, m->device);
    return GRID_E_ARG;
  }
  return GRID_OK;
}

template <class S>
grid_status rollout(const grid_model* m, int B, int H, S dt, const S* q0, const S* qd0, const S* U, const S* K,
                    const S* kff, const S* Qn, const S* QDn, S alpha, S* Q, S* QD, S* Uout, void* stream) {
  grid_status s = check_traj<S>(m, B, H, {q0, qd0, U, Q, QD}, {K, kff, Qn, QDn, Uout});
  if (s != GRID_OK) return s;
  if (K && (!kff || !Qn || !QDn)) { grid_set_error("a policy needs K, kff and the nominal states"); return GRID_E_ARG; }
  if (B == 0) return GRID_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (std::is_same<S, float>::value && m->prec == GRID_MIXED)
    return rollout_dispatch<S, true>(m, B, H, dt, q0, qd0, U, K, kff, Qn, QDn, alpha, Q, QD, Uout, st);
  return rollout_dispatch<S, false>(m, B, H, dt, q0, qd0, U, K, kff, Qn, QDn, alpha, Q, QD, Uout, st);
}

template <class S>
grid_status riccati(const grid_model* m, int B, int H, S dt, const S* Q, const S* QD, const S* U, const S* J,
                    const S* Minv, const S* Qr, const S* QDr, const S* wq, const S* wr, const S* wf, S mu, S* K,
                    S* kff, S* dV, void* stream) {
  grid_status s = check_traj<S>(m, B, H, {Q, QD, U, J, Minv, Qr, QDr, wq, wr, wf, K, kff, dV}, {});
  if (s != GRID_OK) return s;
  if (m->n > 16) { grid_set_error("the Riccati pass supports n <= 16 (n = %d)", m->n); return GRID_E_ARG; }
  if (B == 0) return GRID_OK;
  return launch_riccati<S>(m, B, H, dt, Q, QD, U, J, Minv, Qr, QDr, wq, wr, wf, mu, K, kff, dV,
                           reinterpret_cast<cudaStream_t>(stream));
}

}  // namespace

extern "C" {

grid_status grid_rollout(const grid_model* m, int B, int H, float dt, const float* q0, const float* qd0,
                         const float* U, const float* K, const float* kff, const float* Qnom, const float* QDnom,
                         float alpha, float* Q, float* QD, float* Uout, void* stream) {
  return rollout<float>(m, B, H, dt, q0, qd0, U, K, kff, Qnom, QDnom, alpha, Q, QD, Uout, stream);
}
grid_status grid_rollout_f64(const grid_model* m, int B, int H, double dt, const double* q0, const double* qd0,
                             const double* U, const double* K, const double* kff, const double* Qnom,
                             const double* QDnom, double alpha, double* Q, double* QD, double* Uout, void* stream) {
  return rollout<double>(m, B, H, dt, q0, qd0, U, K, kff, Qnom, QDnom, alpha, Q, QD, Uout, stream);
}
grid_status grid_riccati(const grid_model* m, int B, int H, float dt, const float* Q, const float* QD,
                         const float* U, const float* J, const float* Minv, const float* Qref, const float* QDref,
                         const float* wq, const float* wr, const float* wf, float mu, float* K, float* kff,
                         float* dV, void* stream) {
  return riccati<float>(m, B, H, dt, Q, QD, U, J, Minv, Qref, QDref, wq, wr, wf, mu, K, kff, dV, stream);
}
grid_status grid_riccati_f64(const grid_model* m, int B, int H, double dt, const double* Q, const double* QD,
                             const double* U, const double* J, const double* Minv, const double* Qref,
                             const double* QDref, const double* wq, const double* wr, const double* wf, double mu,
                             double* K, double* kff, double* dV, void* stream) {
  return riccati<double>(m, B, H, dt, Q, QD, U, J, Minv, Qref, QDref, wq, wr, wf, mu, K, kff, dV, stream);
}

}  // extern "C"
