// The dynamics kernel body, device code only: included by grid_launch.cuh and
// compiled at run time by NVRTC for robot-specific topologies (grid_nvrtc.cpp).
#pragma once

#include "grid_internal.h"
#include "grid_phases.cuh"

GRID_HD constexpr int align16(int x) { return (x + 15) & ~15; }

// One CTA: the model head and the lane-count slice of the column schedule are
// staged in shared memory, then each warp loops over tiles of 32/T knot points.
template <class S, int MODE, int T, int CPL, int MAXD, bool MIXED, class Tp>
__device__ __forceinline__ void grid_kernel_body(const ModelDev<S>* __restrict__ gm, int N,
                                                 const S* __restrict__ q, const S* __restrict__ qd,
                                                 const S* __restrict__ x3, const S* __restrict__ x4,
                                                 S* __restrict__ out, S* __restrict__ out2, S* __restrict__ out3) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int cfg = T == 8 ? 0 : (T == 16 ? 1 : 2);
  constexpr int head = align16(model_head_bytes<S>());
  const ModelDev<S>& M = *reinterpret_cast<const ModelDev<S>*>(smem);
  {
    const int4* src = reinterpret_cast<const int4*>(gm);
    int4* dst = reinterpret_cast<int4*>(smem);
    for (int i = threadIdx.x; i < head / 16; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int nsteps = (MODE == MODE_GRAD || MODE == MODE_GRAD_ID) ? M.steps[cfg] : 0;
  const int stride = Tp(M).layout().stride;
  uint32_t* sched = reinterpret_cast<uint32_t*>(smem + head);
  for (int i = threadIdx.x; i < nsteps * T; i += blockDim.x) sched[i] = gm->sched[M.sched_off[cfg] + i];
  S* ws = reinterpret_cast<S*>(smem + head + align16(nsteps * T * 4));
  __syncthreads();
  constexpr int G = 32 / T;
  const int lane32 = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  S* Wwarp = ws + warp * G * stride;
  const int ntiles = (N + G - 1) / G;
  for (int tile = blockIdx.x * wpb + warp; tile < ntiles; tile += gridDim.x * wpb)
    process_tile_t<S, MODE, T, CPL, MAXD, MIXED, Tp>(M, gm, sched, nsteps, Wwarp, lane32, tile * G, N, q, qd, x3,
                                                     x4, out, out2, out3);
}
