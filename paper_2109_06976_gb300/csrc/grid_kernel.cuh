// The dynamics kernel body, device code only: included by grid_launch.cuh and
// compiled at run time by NVRTC for robot-specific topologies (grid_nvrtc.cpp).
#pragma once

#include "grid_internal.h"
#include "grid_phases.cuh"

GRID_HD constexpr int align16(int x) { return (x + 15) & ~15; }

// One CTA: the model head and the lane-count slice of the column schedule are
// staged in shared memory, then each warp loops over tiles of 32/T knot points.
// With KB > 1 the CTA stages the heads of KB models (gm[0 .. KB-1], one per chain
// of a forest run as independent chains; same topology and schedule) and lane
// group g uses model g mod KB.
template <class S, int MODE, int T, int CPL, int MAXD, bool MIXED, class Tp, int KB = 1>
__device__ __forceinline__ void grid_kernel_body(const ModelDev<S>* __restrict__ gm, int N,
                                                 const S* __restrict__ q, const S* __restrict__ qd,
                                                 const S* __restrict__ x3, const S* __restrict__ x4,
                                                 S* __restrict__ out, S* __restrict__ out2, S* __restrict__ out3) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int cfg = T == 8 ? 0 : (T == 16 ? 1 : 2);
  constexpr int head = align16(model_head_bytes<S>());
  static_assert(KB >= 1 && (32 / T) % KB == 0, "every warp tile starts at chain 0");
  for (int b = 0; b < KB; ++b) {
    const int4* src = reinterpret_cast<const int4*>(gm + b);
    int4* dst = reinterpret_cast<int4*>(smem + b * head);
    for (int i = threadIdx.x; i < head / 16; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const ModelDev<S>& M0 = *reinterpret_cast<const ModelDev<S>*>(smem);
  const int nsteps = (MODE == MODE_GRAD || MODE == MODE_GRAD_ID) ? M0.steps[cfg] : 0;
  const int stride = Tp(M0).layout().stride;
  uint32_t* sched = reinterpret_cast<uint32_t*>(smem + KB * head);
  for (int i = threadIdx.x; i < nsteps * T; i += blockDim.x) sched[i] = gm->sched[M0.sched_off[cfg] + i];
  S* ws = reinterpret_cast<S*>(smem + KB * head + align16(nsteps * T * 4));
  __syncthreads();
  constexpr int G = 32 / T;
  const int lane32 = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int mb = KB > 1 ? (lane32 / T) % KB : 0;
  const ModelDev<S>& M = *reinterpret_cast<const ModelDev<S>*>(smem + mb * head);
  S* Wwarp = ws + warp * G * stride;
  const int ntiles = (N + G - 1) / G;
  for (int tile = blockIdx.x * wpb + warp; tile < ntiles; tile += gridDim.x * wpb)
    process_tile_t<S, MODE, T, CPL, MAXD, MIXED, Tp>(M, gm + mb, sched, nsteps, Wwarp, lane32, tile * G, N, q, qd,
                                                     x3, x4, out, out2, out3);
}
