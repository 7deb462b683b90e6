// Kernel template and launcher (included by the per-precision translation units).
//
// Mapping: T lanes (8, 16 or 32) of a warp cooperate on one knot point; a warp
// holds 32/T knot points and every group of the warp runs the same robot in
// lockstep, so all synchronisation inside a tile is __syncwarp(). Warps are
// independent and loop over tiles of knot points (persistent grid sized from
// the occupancy calculator). Each knot point owns a shared-memory workspace
// (KnotLayout); the CTA holds one copy of the robot model.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <type_traits>

#include "grid_internal.h"
#include "grid_kernel.cuh"

// ---------------------------------------------------------------- kernel
template <class S, int MODE, int T, int CPL, int MAXD, bool MIXED, int CHAIN_N>
__global__ void __launch_bounds__(128, CHAIN_N > 0 ? 4 : 1) grid_kernel(const ModelDev<S>* __restrict__ gm, int N,
                                                   const S* __restrict__ q, const S* __restrict__ qd,
                                                   const S* __restrict__ x3, const S* __restrict__ x4,
                                                   S* __restrict__ out, S* __restrict__ out2,
                                                   S* __restrict__ out3) {
  grid_kernel_body<S, MODE, T, CPL, MAXD, MIXED, topo_for<S, MODE, CHAIN_N>>(gm, N, q, qd, x3, x4, out, out2, out3);
}

// A forest of KB chains of L bodies run as KB independent chains (BranchTopo):
// N counts the virtual knot points (knot points x KB); gm is the array of the
// KB chain models. In FP32 five CTAs per SM fit without spills (at most 102
// registers; measured +3 % on the 12-DoF tree against four); FP64 keeps four.
template <class S, int MODE, int T, int CPL, int MAXD, bool MIXED, int L, int KB>
__global__ void __launch_bounds__(128, sizeof(S) == 4 ? 5 : 4) grid_branch_kernel(const ModelDev<S>* __restrict__ gm, int N,
                                                  const S* __restrict__ q, const S* __restrict__ qd,
                                                  const S* __restrict__ x3, const S* __restrict__ x4,
                                                  S* __restrict__ out, S* __restrict__ out2,
                                                  S* __restrict__ out3) {
  grid_kernel_body<S, MODE, T, CPL, MAXD, MIXED, BranchTopo<S, MODE, L, KB>, KB>(gm, N, q, qd, x3, x4, out, out2,
                                                                                   out3);
}

// ---------------------------------------------------------------- launcher
constexpr int kMaxWarps = 4;    // warps per CTA (matches __launch_bounds__)

struct DevInfo {
  int nsm = 0, smem_optin = 0;
};

static inline DevInfo dev_info(int dev) {
  static DevInfo cache[64];
  static std::atomic<int> ready[64];
  if (dev < 0 || dev >= 64) return DevInfo{};
  if (!ready[dev].load()) {
    DevInfo d;
    cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cache[dev] = d;
    ready[dev].store(1);
  }
  return cache[dev];
}

// KB > 1: the branch kernel for a forest of KB chains of CHAIN_N bodies; hm is
// the first chain's host model, dm the device array of the KB chain models and N
// the number of virtual knot points.
template <class S, int MODE, int T, int CPL, int MAXD, bool MIXED, int CHAIN_N = 0, int KB = 1>
grid_status launch_t(const grid_model* m, const ModelDev<S>* hm, const ModelDev<S>* dm, int N,
                     const S* q, const S* qd, const S* x3, const S* x4, S* out, S* out2, S* out3,
                     cudaStream_t st) {
  static_assert(KB == 1 || CHAIN_N > 0, "branches are chains");
  auto kern = [] {
    if constexpr (KB > 1) return grid_branch_kernel<S, MODE, T, CPL, MAXD, MIXED, CHAIN_N, KB>;
    else return grid_kernel<S, MODE, T, CPL, MAXD, MIXED, CHAIN_N>;
  }();
  if constexpr (CHAIN_N > 0) {
    // the compile-time layout must be the one the host built for this model
    constexpr int NB = CHAIN_N % 100;
    if (hm->n != NB || ChainTopo<S, MODE, NB>::layout().stride != layout_of<MODE>(*hm).stride ||
        (CHAIN_N > 100) != (hm->ld != hm->n)) {
      grid_set_error("chain kernel for %d bodies does not match the model", NB);
      return GRID_E_TOPOLOGY;
    }
  } else if constexpr (CHAIN_N < 0) {
    using F = ForestTopo<S, MODE, -CHAIN_N / 100, -CHAIN_N % 100>;
    if (hm->n != F::n() || F::layout().stride != layout_of<MODE>(*hm).stride) {
      grid_set_error("forest kernel does not match the model");
      return GRID_E_TOPOLOGY;
    }
  }
  constexpr int cfg = T == 8 ? 0 : (T == 16 ? 1 : 2);
  constexpr int G = 32 / T;
  const int nsteps = (MODE == MODE_GRAD || MODE == MODE_GRAD_ID) ? hm->steps[cfg] : 0;
  const DevInfo di = dev_info(m->device);
  const size_t fixed = KB * align16(model_head_bytes<S>()) + align16(nsteps * T * 4);
  const size_t per_warp = (size_t)G * layout_of<MODE>(*hm).stride * sizeof(S);
  // Opt in to large dynamic shared memory once per instantiation.
  static std::atomic<int> opted{0};
  cudaError_t err = cudaSuccess;
  if (!opted.load()) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)di.smem_optin);
    if (err != cudaSuccess) {
      grid_set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(err));
      return GRID_E_CUDA;
    }
    opted.store(1);
  }
  // Warps per CTA: the count that keeps the most warps resident per SM (ties go
  // to larger CTAs, which share one copy of the model among more warps). The
  // choice is cached per instantiation and workspace size.
  static std::atomic<unsigned long long> cached{0};
  int warps = 0, per_sm = 0, best = 0;
  const unsigned long long c0 = cached.load();
  if (c0 && (c0 >> 16) == (unsigned long long)(fixed + per_warp)) {
    warps = (int)((c0 >> 8) & 0xff);
    per_sm = (int)(c0 & 0xff);
  } else {
    for (int w = kMaxWarps; w >= 1; --w) {
      const size_t sm_w = fixed + w * per_warp;
      if (sm_w > (size_t)di.smem_optin) continue;
      int b = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 32 * w, sm_w);
      if (b * w > best) { best = b * w; warps = w; per_sm = b; }
    }
    if (warps) cached.store(((unsigned long long)(fixed + per_warp) << 16) | (warps << 8) | (per_sm & 0xff));
  }
  if (warps == 0) {
    grid_set_error("knot workspace needs %zu B of shared memory per warp (limit %d); use more lanes",
                   fixed + per_warp, di.smem_optin);
    return GRID_E_ARG;
  }
  const size_t smem = fixed + warps * per_warp;
  const int threads = 32 * warps;
  if (m->ctas_opt > 0 && m->ctas_opt < per_sm) per_sm = m->ctas_opt;
  const long tiles = (N + G - 1) / G;
  const long ctas_needed = (tiles + warps - 1) / warps;
  const int grid = (int)std::min<long>(ctas_needed, (long)di.nsm * per_sm);
  kern<<<grid, threads, smem, st>>>(dm, N, q, qd, x3, x4, out, out2, out3);
  err = cudaGetLastError();
  if (err != cudaSuccess) {
    grid_set_error("kernel launch: %s", cudaGetErrorString(err));
    return GRID_E_CUDA;
  }
  return GRID_OK;
}

template <class S, int MODE, int T, int CPL, bool MIXED>
grid_status launch_d(const grid_model* m, const ModelDev<S>* hm, const ModelDev<S>* dm, int N, const S* q,
                     const S* qd, const S* x3, const S* x4, S* out, S* out2, S* out3, cudaStream_t st) {
  if ((MODE == MODE_GRAD || MODE == MODE_GRAD_ID) && hm->maxd > 8)
    return launch_t<S, MODE, T, CPL, 32, MIXED>(m, hm, dm, N, q, qd, x3, x4, out, out2, out3, st);
  return launch_t<S, MODE, T, CPL, 8, MIXED>(m, hm, dm, N, q, qd, x3, x4, out, out2, out3, st);
}

// Serial chains of 2 .. kChainMaxN bodies run a kernel compiled for their
// length (grid_chain.cu); 8 lanes per knot point.
constexpr int kChainMaxN = 8;
template <class S, int MODE>
grid_status launch_chain(const grid_model* m, const ModelDev<S>* hm, const ModelDev<S>* dm, int N, const S* q,
                         const S* qd, const S* x3, const S* x4, S* out, S* out2, S* out3, cudaStream_t st);
// Gradient of FD of a serial chain of 2 .. 8 revolute bodies with one lane per
// knot point (grid_lane_chain.cu): the throughput form for large batches. With
// slot non-NULL the chain is a component of a robot of ld joints per knot point
// whose body i is caller joint slot[i] (a leg of a forest, a part).
grid_status launch_lane_chain(const grid_model* m, const ModelDev<float>* hm, int ld, const int* slot, int N,
                              const float* q, const float* qd, const float* tau, float* J, float* qdd,
                              float* Minv, cudaStream_t st);
// FD and the vector-Jacobian product through FD in the same form
// (grid_lane_chain_fdv.cu): qdd; dL/dq, dL/dqd, dL/dtau for gbar = dL/dqdd.
grid_status launch_lane_chain_fd(const grid_model* m, const ModelDev<float>* hm, int ld, const int* slot, int N,
                                 const float* q, const float* qd, const float* tau, float* qdd, cudaStream_t st);
grid_status launch_lane_chain_vjp(const grid_model* m, const ModelDev<float>* hm, int ld, const int* slot, int N,
                                  const float* q, const float* qd, const float* tau, const float* gbar, float* dq,
                                  float* dqd, float* dtau, cudaStream_t st);
// RNEA (qdd NULL for zero), M^-1 and the gradient of ID in the same form
// (grid_lane_chain_id.cu); a placed chain writes its whole rows of M^-1 or D.
grid_status launch_lane_chain_rnea(const grid_model* m, const ModelDev<float>* hm, int ld, const int* slot, int N,
                                   const float* q, const float* qd, const float* qdd, float* tau, cudaStream_t st);
grid_status launch_lane_chain_minv(const grid_model* m, const ModelDev<float>* hm, int ld, const int* slot, int N,
                                   const float* q, float* Minv, cudaStream_t st);
grid_status launch_lane_chain_grad_id(const grid_model* m, const ModelDev<float>* hm, int ld, const int* slot,
                                      int N, const float* q, const float* qd, const float* qdd, float* D,
                                      cudaStream_t st);
// Batches from this many knot points up take the one-lane-per-knot-point chain
// kernel by default (below, the 8-lane kernel has the shorter latency).
constexpr int kLaneChainMinN = 32768;
// The same for a chain that is a part placed in a robot's arrays (grid_chain_part.cu).
template <class S, int MODE>
grid_status launch_chain_part(const grid_model* m, const ModelDev<S>* hm, const ModelDev<S>* dm, int N,
                              const S* q, const S* qd, const S* x3, const S* x4, S* out, S* out2, S* out3,
                              cudaStream_t st);
// Kernels compiled at run time for the model's topology (grid_nvrtc.cpp).
template <class S>
grid_status grid_gen_launch(grid_model* m, const ModelDev<S>* hm, const ModelDev<S>* dm, int N, const S* q,
                            const S* qd, const S* tau, S* J, S* qdd, S* Minv, int T, int CPL, int MAXD, int nsm,
                            int smem_optin, cudaStream_t st);

// The parts of a robot at once on small batches (grid_capi.cu): fork the caller's
// stream into one stream per part (holds the model's lock until the join), then
// join them into the caller's stream again.
grid_status grid_parts_fork(const grid_model* m, cudaStream_t caller, cudaStream_t* streams);
grid_status grid_parts_join(const grid_model* m, cudaStream_t caller);

// Forests of K equal chains (grid_forest.cu), compiled for a few shapes.
bool forest_compiled(int k, int l);
template <class S, int MODE>
grid_status launch_forest(const grid_model* m, const ModelDev<S>* hm, const ModelDev<S>* dm, int N, const S* q,
                          const S* qd, const S* x3, const S* x4, S* out, S* out2, S* out3, cudaStream_t st);

// The kernel for one model (the robot, or one of its parts): the lane count T
// (option or by size), the M^-1 columns per lane, run-time specialisation.
template <class S, int MODE, bool MIXED>
grid_status dispatch_model(const grid_model* m, const ModelDev<S>* hm, const ModelDev<S>* dm, int T, int N,
                           const S* q, const S* qd, const S* x3, const S* x4, S* out, S* out2, S* out3,
                           cudaStream_t st) {
  const int n = hm->n;
  // Default lanes: 8 up to 12 bodies, 16 up to 16, else 32 (throughput; above
  // 16 bodies one warp per knot point halves the workspace per warp, measured on
  // the 30-DoF tree and its 20-body torso-and-arms component). A batch smaller
  // than two knot points per SM is latency-bound: for more bodies than 8 lanes,
  // one warp per knot point then shortens the parallel phases (measured for the
  // 12- and 30-DoF trees; up to 8 bodies, 8 lanes stay faster).
  if (T == 0) T = (n > 8 && N <= 2 * dev_info(m->device).nsm) ? 32 : (n <= 12 ? 8 : (n <= 16 ? 16 : 32));
  const int cpl = (n + T - 1) / T;
  if constexpr (MODE == MODE_GRAD && !MIXED) {
    if (m->specialize_opt == 2 && (T == 8 || T == 16 || T == 32)) {
      const int c = T == 8 ? (cpl <= 1 ? 1 : (cpl <= 2 ? 2 : 4)) : (T == 16 ? (cpl <= 1 ? 1 : 2) : 1);
      const DevInfo di = dev_info(m->device);
      return grid_gen_launch<S>(const_cast<grid_model*>(m), hm, dm, N, q, qd, x3, out, out2, out3, T, c,
                                hm->maxd > 8 ? 32 : 8, di.nsm, di.smem_optin, st);
    }
  }
  if (T == 8) {
    if (cpl <= 1) return launch_d<S, MODE, 8, 1, MIXED>(m, hm, dm, N, q, qd, x3, x4, out, out2, out3, st);
    if (cpl <= 2) return launch_d<S, MODE, 8, 2, MIXED>(m, hm, dm, N, q, qd, x3, x4, out, out2, out3, st);
    return launch_d<S, MODE, 8, 4, MIXED>(m, hm, dm, N, q, qd, x3, x4, out, out2, out3, st);
  }
  if (T == 16) {
    if (cpl <= 1) return launch_d<S, MODE, 16, 1, MIXED>(m, hm, dm, N, q, qd, x3, x4, out, out2, out3, st);
    return launch_d<S, MODE, 16, 2, MIXED>(m, hm, dm, N, q, qd, x3, x4, out, out2, out3, st);
  }
  if (T == 32) return launch_d<S, MODE, 32, 1, MIXED>(m, hm, dm, N, q, qd, x3, x4, out, out2, out3, st);
  grid_set_error("lanes option %d not in {0, 8, 16, 32}", T);
  return GRID_E_ARG;
}

// Picks the kernels for a model: the chain or forest kernels compiled for its
// topology, its base components one after another (parts), or dispatch_model.
template <class S, int MODE, bool MIXED>
grid_status dispatch(const grid_model* m, int N, const S* q, const S* qd, const S* x3, const S* x4,
                     S* out, S* out2, S* out3, cudaStream_t st) {
  const ModelDev<S>* hm;
  const ModelDev<S>* dm;
  if constexpr (std::is_same<S, float>::value) { hm = m->host_f; dm = m->dev_f; }
  else { hm = m->host_d; dm = m->dev_d; }
  // lanes 1: one lane per knot point where that kernel exists (the gradient of
  // FD of FP32 serial chains), automatic elsewhere
  const int T = m->lanes_opt == 1 ? 0 : m->lanes_opt;
  const int n = hm->n;
  if constexpr (MODE != MODE_GRAD && !MIXED && std::is_same<S, float>::value) {
    // RNEA, M^-1, FD, the gradient of ID and the vector-Jacobian product of chains
    // and of a forest's legs, one lane per knot point (each leg writes its joints'
    // entries of the vector outputs and its whole rows of the matrix outputs: its
    // blocks and the zeros beside them)
    bool lane1 = m->specialize_opt && (m->lanes_opt == 1 || (m->lanes_opt == 0 && N >= kLaneChainMinN));
    if (lane1 && m->lanes_opt == 0) {
      cudaPointerAttributes pa{};
      if (cudaPointerGetAttributes(&pa, out) != cudaSuccess) {
        cudaGetLastError();
        lane1 = false;
      } else if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) {
        lane1 = false;
      }
    }
    auto one = [&](const ModelDev<float>* mh, const int* slot) {
      if constexpr (MODE == MODE_FD) return launch_lane_chain_fd(m, mh, n, slot, N, q, qd, x3, out, st);
      else if constexpr (MODE == MODE_VJP)
        return launch_lane_chain_vjp(m, mh, n, slot, N, q, qd, x3, x4, out, out2, out3, st);
      else if constexpr (MODE == MODE_RNEA) return launch_lane_chain_rnea(m, mh, n, slot, N, q, qd, x3, out, st);
      else if constexpr (MODE == MODE_MINV) return launch_lane_chain_minv(m, mh, n, slot, N, q, out, st);
      else return launch_lane_chain_grad_id(m, mh, n, slot, N, q, qd, x3, out, st);
    };
    if (lane1 && m->chain && n >= 2 && n <= kChainMaxN) return one(hm, nullptr);
    if (lane1 && m->forest_k > 1 && m->branches == m->forest_k && m->forest_l >= 2 && m->forest_l <= kChainMaxN &&
        n <= 32) {
      int slot[kChainMaxN];
      for (int c = 0; c < m->forest_k; ++c) {
        for (int i = 0; i < m->forest_l; ++i) slot[i] = c * m->forest_l + i;
        const grid_status r = one(&m->br_host_f[c], slot);
        if (r != GRID_OK) return r;
      }
      return GRID_OK;
    }
  }
  if constexpr (MODE == MODE_GRAD && !MIXED && std::is_same<S, float>::value) {
    // (by default not for outputs in host memory: its scattered per-lane stores
    // over the host link measured 2.6e7 against 2.2e8 knot-points/s for the
    // 8-lane kernel's row-wise stores, 7-DoF chain, 2,097,152 knot points)
    bool lane1 = m->specialize_opt && (m->lanes_opt == 1 || (m->lanes_opt == 0 && N >= kLaneChainMinN));
    if (lane1 && m->lanes_opt == 0) {
      cudaPointerAttributes pa{};
      if (cudaPointerGetAttributes(&pa, out) != cudaSuccess) {
        cudaGetLastError();
        lane1 = false;
      } else if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) {
        lane1 = false;
      }
    }
    if (lane1 && m->chain && n >= 2 && n <= kChainMaxN)
      return launch_lane_chain(m, hm, n, nullptr, N, q, qd, x3, out, out2, out3, st);
    // a forest with one model per chain: each chain (a leg) in turn, one lane per
    // (knot point, leg), writing its whole rows of J and M^-1 (its blocks and the
    // zeros beside them, from blocks staged per warp) and its entries of qdd
    if (lane1 && m->forest_k > 1 && m->branches == m->forest_k && m->forest_l >= 2 && m->forest_l <= kChainMaxN &&
        n <= 32) {
      int slot[kChainMaxN];
      for (int c = 0; c < m->forest_k; ++c) {
        for (int i = 0; i < m->forest_l; ++i) slot[i] = c * m->forest_l + i;
        const grid_status r =
            launch_lane_chain(m, &m->br_host_f[c], n, slot, N, q, qd, x3, out, out2, out3, st);
        if (r != GRID_OK) return r;
      }
      return GRID_OK;
    }
  }
  if constexpr (MODE == MODE_GRAD && !MIXED) {
    if (m->chain && m->specialize_opt && (T == 0 || T == 8) && n >= 2 && n <= kChainMaxN)
      return launch_chain<S, MODE>(m, hm, dm, N, q, qd, x3, x4, out, out2, out3, st);
    if (m->forest_k > 1 && m->specialize_opt && T == 0 && forest_compiled(m->forest_k, m->forest_l))
      return launch_forest<S, MODE>(m, hm, dm, N, q, qd, x3, x4, out, out2, out3, st);
  }
  if constexpr (MODE == MODE_GRAD) {
    // Base components that differ (a humanoid's torso with its arms, and its
    // legs) share nothing through the fixed base: each runs as a problem of its
    // own, in the kernel for its size and topology, and writes its rows of J
    // (and of M^-1 and qdd). The parts run at the same time on streams of their
    // own, forked from and joined into the caller's stream: small batches then
    // take the time of the largest part (30-DoF tree, one knot point: 60 to 56 us),
    // and mid-size ones do not wait for parts one after another (1024 knot points:
    // 93 us in sequence against 74 us for the whole robot).
    if (m->nparts > 0 && m->pexec && m->specialize_opt && T == 0) {
      cudaStream_t ps[GRID_MAX_DOF];
      const grid_status f = grid_parts_fork(m, st, ps);
      if (f != GRID_OK) return f;
      grid_status r = GRID_OK;
      for (int p = 0; r == GRID_OK && p < m->nparts; ++p) {
        const grid_part& P = m->parts[p];
        const ModelDev<S>* ph;
        const ModelDev<S>* pd;
        if constexpr (std::is_same<S, float>::value) { ph = P.host_f; pd = P.dev_f; }
        else { ph = P.host_d; pd = P.dev_d; }
        const cudaStream_t s = ps[p];
        const bool lane1 = m->lanes_opt == 1 || N >= kLaneChainMinN;
        if (!MIXED && P.chain && P.n >= 2 && P.n <= kChainMaxN && std::is_same<S, float>::value && lane1 &&
            ph->ld <= 32) {
          if constexpr (std::is_same<S, float>::value)
            r = launch_lane_chain(m, ph, ph->ld, ph->gslot, N, q, qd, x3, out, out2, out3, s);
        } else if (!MIXED && P.chain && P.n >= 2 && P.n <= kChainMaxN) {
          r = launch_chain_part<S, MODE>(m, ph, pd, N, q, qd, x3, x4, out, out2, out3, s);
        } else {
          r = dispatch_model<S, MODE, MIXED>(m, ph, pd, 0, N, q, qd, x3, x4, out, out2, out3, s);
        }
      }
      const grid_status j = grid_parts_join(m, st);
      return r == GRID_OK ? j : r;
    }
  }
  return dispatch_model<S, MODE, MIXED>(m, hm, dm, T, N, q, qd, x3, x4, out, out2, out3, st);
}


#define GRID_INSTANTIATE(S, MIXED)                                                                   \
  template grid_status dispatch<S, MODE_RNEA, MIXED>(const grid_model*, int, const S*, const S*,     \
                                                     const S*, const S*, S*, S*, S*, cudaStream_t);  \
  template grid_status dispatch<S, MODE_MINV, MIXED>(const grid_model*, int, const S*, const S*,     \
                                                     const S*, const S*, S*, S*, S*, cudaStream_t);  \
  template grid_status dispatch<S, MODE_FD, MIXED>(const grid_model*, int, const S*, const S*,       \
                                                   const S*, const S*, S*, S*, S*, cudaStream_t);  \
  template grid_status dispatch<S, MODE_GRAD, MIXED>(const grid_model*, int, const S*, const S*,     \
                                                     const S*, const S*, S*, S*, S*, cudaStream_t);  \
  template grid_status dispatch<S, MODE_VJP, MIXED>(const grid_model*, int, const S*, const S*,      \
                                                    const S*, const S*, S*, S*, S*, cudaStream_t);   \
  template grid_status dispatch<S, MODE_GRAD_ID, MIXED>(const grid_model*, int, const S*, const S*,  \
                                                        const S*, const S*, S*, S*, S*, cudaStream_t);
