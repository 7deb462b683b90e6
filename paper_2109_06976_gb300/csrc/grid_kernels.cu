// Batched rigid-body dynamics kernels for sm_103a: RNEA, direct M^-1, FD and
// the analytical gradient of FD (GRiD, Sec. IV-B; Alg. 1 / Alg. 2).
//
// Mapping. T lanes (8, 16 or 32) of a warp cooperate on one knot point; a warp
// holds 32/T knot points and every group of the warp runs the same robot in
// lockstep, so all synchronisation is __syncwarp(). Warps are independent and
// loop over tiles of knot points (persistent grid). Each knot point owns a
// workspace in shared memory (layout in KnotLayout); the CTA keeps one copy of
// the robot model.
//
// Phases for one knot point (all in the internal depth-first numbering):
//  B1 joint transforms X_i(q_i)                      lanes over bodies
//  B2 RNEA forward/backward sweeps (Sec. IV-B)       lanes over the 6 components
//  B3 direct M^-1 (articulated-inertia recursion)    lanes over 6x6 entries / columns
//  B4 qdd = M^-1 (tau - c)                           lanes over rows
//  B5 RNEA at qdd: a, f, accumulated F                lanes over components
//  B6 per-body case terms of Alg. 2 and the ancestor subspaces s_i^(k)
//  C  derivative columns (Alg. 1 / Alg. 2 forward pass; backward pass by
//     ancestor dot products): lanes run host-balanced schedules of
//     root-to-leaf paths, state in registers
//  D  J = -M^-1 dc                                   lanes over outputs
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <initializer_list>
#include <string>
#include <type_traits>

#include "grid_internal.h"
#include "spatial.cuh"

#include "grid_phases.cuh"

namespace {

// ---------------------------------------------------------------- kernel
__host__ __device__ constexpr int align16(int x) { return (x + 15) & ~15; }

template <class S, int MODE, int T, int MAXD, bool MIXED>
__global__ void __launch_bounds__(128) grid_kernel(const ModelDev<S>* __restrict__ gm, int N,
                                                   const S* __restrict__ q, const S* __restrict__ qd,
                                                   const S* __restrict__ x3, S* __restrict__ out,
                                                   S* __restrict__ out2) {
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
  const int nsteps = (MODE == MODE_GRAD) ? M.steps[cfg] : 0;
  uint32_t* sched = reinterpret_cast<uint32_t*>(smem + head);
  for (int i = threadIdx.x; i < nsteps * T; i += blockDim.x) sched[i] = gm->sched[M.sched_off[cfg] + i];
  S* ws = reinterpret_cast<S*>(smem + head + align16(nsteps * T * 4));
  __syncthreads();
  constexpr int G = 32 / T;
  const int lane32 = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  S* Wwarp = ws + warp * G * M.L.stride;
  const int ntiles = (N + G - 1) / G;
  for (int tile = blockIdx.x * wpb + warp; tile < ntiles; tile += gridDim.x * wpb)
    process_tile<S, MODE, T, MAXD, MIXED>(M, sched, nsteps, Wwarp, lane32, tile * G, N, q, qd, x3, out, out2);
}

// ---------------------------------------------------------------- launcher
constexpr int kMaxWarps = 4;    // warps per CTA (matches __launch_bounds__)

struct DevInfo {
  int nsm = 0, smem_optin = 0;
};

DevInfo dev_info(int dev) {
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

template <class S, int MODE, int T, int MAXD, bool MIXED>
grid_status launch_t(const grid_model* m, const ModelDev<S>* hm, const ModelDev<S>* dm, int N,
                     const S* q, const S* qd, const S* x3, S* out, S* out2, cudaStream_t st) {
  auto kern = grid_kernel<S, MODE, T, MAXD, MIXED>;
  constexpr int cfg = T == 8 ? 0 : (T == 16 ? 1 : 2);
  constexpr int G = 32 / T;
  const int nsteps = (MODE == MODE_GRAD) ? hm->steps[cfg] : 0;
  const DevInfo di = dev_info(m->device);
  const size_t fixed = align16(model_head_bytes<S>()) + align16(nsteps * T * 4);
  const size_t per_warp = (size_t)G * hm->L.stride * sizeof(S);
  int warps = kMaxWarps;
  while (warps > 1 && fixed + warps * per_warp > (size_t)di.smem_optin) --warps;
  const size_t smem = fixed + warps * per_warp;
  if (smem > (size_t)di.smem_optin) {
    grid_set_error("knot workspace needs %zu B of shared memory (limit %d); use more lanes",
                   smem, di.smem_optin);
    return GRID_E_ARG;
  }
  // Opt in to large dynamic shared memory once per instantiation and size.
  static std::atomic<size_t> opted{0};
  cudaError_t err = cudaSuccess;
  if (smem > opted.load()) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)di.smem_optin);
    if (err != cudaSuccess) {
      grid_set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(err));
      return GRID_E_CUDA;
    }
    opted.store((size_t)di.smem_optin);
  }
  const int threads = 32 * warps;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (per_sm < 1) {
    grid_set_error("kernel does not fit on an SM (%zu B shared per CTA)", smem);
    return GRID_E_CUDA;
  }
  if (m->ctas_opt > 0 && m->ctas_opt < per_sm) per_sm = m->ctas_opt;
  const long tiles = (N + G - 1) / G;
  const long ctas_needed = (tiles + warps - 1) / warps;
  const int grid = (int)std::min<long>(ctas_needed, (long)di.nsm * per_sm);
  kern<<<grid, threads, smem, st>>>(dm, N, q, qd, x3, out, out2);
  err = cudaGetLastError();
  if (err != cudaSuccess) {
    grid_set_error("kernel launch: %s", cudaGetErrorString(err));
    return GRID_E_CUDA;
  }
  return GRID_OK;
}

template <class S, int MODE, bool MIXED>
grid_status dispatch(const grid_model* m, int N, const S* q, const S* qd, const S* x3, S* out, S* out2,
                     cudaStream_t st) {
  const ModelDev<S>* hm;
  const ModelDev<S>* dm;
  if constexpr (std::is_same<S, float>::value) { hm = m->host_f; dm = m->dev_f; }
  else { hm = m->host_d; dm = m->dev_d; }
  int T = m->lanes_opt;
  if (T == 0) T = hm->n <= 12 ? 8 : (hm->n <= 20 ? 16 : 32);
  const bool deep = hm->maxd > 8;
#define GRID_CASE(TT)                                                                              \
  if (T == TT) {                                                                                   \
    if (deep) return launch_t<S, MODE, TT, 32, MIXED>(m, hm, dm, N, q, qd, x3, out, out2, st);     \
    return launch_t<S, MODE, TT, 8, MIXED>(m, hm, dm, N, q, qd, x3, out, out2, st);                \
  }
  GRID_CASE(8)
  GRID_CASE(16)
  GRID_CASE(32)
#undef GRID_CASE
  grid_set_error("lanes option %d not in {0, 8, 16, 32}", T);
  return GRID_E_ARG;
}

template <class S>
grid_status check_args(const grid_model* m, int N, std::initializer_list<const void*> must,
                       std::initializer_list<const void*> may) {
  if (!m) { grid_set_error("null model"); return GRID_E_ARG; }
  if (N < 0) { grid_set_error("N = %d < 0", N); return GRID_E_ARG; }
  for (const void* p : must) {
    if (!p && N > 0) { grid_set_error("null state or output pointer"); return GRID_E_ARG; }
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

template <class S, int MODE>
grid_status run(const grid_model* m, int N, const S* q, const S* qd, const S* x3, S* out, S* out2,
                void* stream) {
  if (N == 0) return GRID_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (std::is_same<S, float>::value && m->prec == GRID_MIXED)
    return dispatch<S, MODE, true>(m, N, q, qd, x3, out, out2, st);
  return dispatch<S, MODE, false>(m, N, q, qd, x3, out, out2, st);
}

}  // namespace

// ---------------------------------------------------------------- C-ABI
extern "C" {

grid_status grid_create(int n, const int* parent, const double* axis, const double* X_tree,
                        const double* inertia, const double* gravity, grid_precision prec,
                        grid_model** out) {
  if (!out) { grid_set_error("grid_create: null output handle"); return GRID_E_ARG; }
  *out = nullptr;
  if (prec != GRID_FP32 && prec != GRID_MIXED && prec != GRID_FP64) {
    grid_set_error("grid_create: bad precision %d", (int)prec);
    return GRID_E_ARG;
  }
  grid_model* m = new grid_model();
  m->n = n;
  m->prec = prec == GRID_FP64 ? GRID_FP32 : prec;
  m->lanes_opt = 0;
  m->ctas_opt = 0;
  m->host_f = new ModelDev<float>();
  m->host_d = new ModelDev<double>();
  grid_status s = grid_build_model(n, parent, axis, X_tree, inertia, gravity, m->host_f, m->host_d);
  if (s != GRID_OK) { delete m->host_f; delete m->host_d; delete m; return s; }
  cudaGetDevice(&m->device);
  cudaError_t e1 = cudaMalloc(&m->dev_f, sizeof(ModelDev<float>));
  cudaError_t e2 = cudaMalloc(&m->dev_d, sizeof(ModelDev<double>));
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    grid_set_error("grid_create: cudaMalloc: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    if (e1 == cudaSuccess) cudaFree(m->dev_f);
    if (e2 == cudaSuccess) cudaFree(m->dev_d);
    delete m->host_f; delete m->host_d; delete m;
    return GRID_E_NOMEM;
  }
  e1 = cudaMemcpy(m->dev_f, m->host_f, sizeof(ModelDev<float>), cudaMemcpyHostToDevice);
  e2 = cudaMemcpy(m->dev_d, m->host_d, sizeof(ModelDev<double>), cudaMemcpyHostToDevice);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    grid_set_error("grid_create: cudaMemcpy: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    cudaFree(m->dev_f); cudaFree(m->dev_d);
    delete m->host_f; delete m->host_d; delete m;
    return GRID_E_CUDA;
  }
  *out = m;
  return GRID_OK;
}

grid_status grid_destroy(grid_model* m) {
  if (!m) return GRID_OK;
  cudaDeviceSynchronize();
  cudaFree(m->dev_f);
  cudaFree(m->dev_d);
  delete m->host_f;
  delete m->host_d;
  delete m;
  return GRID_OK;
}

int grid_model_dof(const grid_model* m) { return m ? m->n : 0; }

grid_status grid_set_option(grid_model* m, const char* key, int value) {
  if (!m || !key) { grid_set_error("grid_set_option: null argument"); return GRID_E_ARG; }
  std::string k(key);
  if (k == "lanes") {
    if (value != 0 && value != 8 && value != 16 && value != 32) {
      grid_set_error("lanes must be 0, 8, 16 or 32"); return GRID_E_ARG;
    }
    m->lanes_opt = value;
  } else if (k == "precision") {
    if (value != GRID_FP32 && value != GRID_MIXED) {
      grid_set_error("precision must be GRID_FP32 or GRID_MIXED"); return GRID_E_ARG;
    }
    m->prec = (grid_precision)value;
  } else if (k == "ctas_per_sm") {
    if (value < 0) { grid_set_error("ctas_per_sm must be >= 0"); return GRID_E_ARG; }
    m->ctas_opt = value;
  } else {
    grid_set_error("unknown option '%s'", key);
    return GRID_E_ARG;
  }
  return GRID_OK;
}

grid_status grid_rnea(const grid_model* m, int N, const float* q, const float* qd, const float* qdd,
                      float* tau, void* stream) {
  grid_status s = check_args<float>(m, N, {q, qd, tau}, {qdd});
  if (s != GRID_OK) return s;
  return run<float, MODE_RNEA>(m, N, q, qd, qdd, tau, nullptr, stream);
}
grid_status grid_minv(const grid_model* m, int N, const float* q, float* Minv, void* stream) {
  grid_status s = check_args<float>(m, N, {q, Minv}, {});
  if (s != GRID_OK) return s;
  return run<float, MODE_MINV>(m, N, q, nullptr, nullptr, Minv, nullptr, stream);
}
grid_status grid_fd(const grid_model* m, int N, const float* q, const float* qd, const float* tau,
                    float* qdd, void* stream) {
  grid_status s = check_args<float>(m, N, {q, qd, tau, qdd}, {});
  if (s != GRID_OK) return s;
  return run<float, MODE_FD>(m, N, q, qd, tau, qdd, nullptr, stream);
}
grid_status grid_grad_fd(const grid_model* m, int N, const float* q, const float* qd, const float* tau,
                         float* J, float* qdd, void* stream) {
  grid_status s = check_args<float>(m, N, {q, qd, tau, J}, {qdd});
  if (s != GRID_OK) return s;
  return run<float, MODE_GRAD>(m, N, q, qd, tau, J, qdd, stream);
}
grid_status grid_rnea_f64(const grid_model* m, int N, const double* q, const double* qd,
                          const double* qdd, double* tau, void* stream) {
  grid_status s = check_args<double>(m, N, {q, qd, tau}, {qdd});
  if (s != GRID_OK) return s;
  return run<double, MODE_RNEA>(m, N, q, qd, qdd, tau, nullptr, stream);
}
grid_status grid_minv_f64(const grid_model* m, int N, const double* q, double* Minv, void* stream) {
  grid_status s = check_args<double>(m, N, {q, Minv}, {});
  if (s != GRID_OK) return s;
  return run<double, MODE_MINV>(m, N, q, nullptr, nullptr, Minv, nullptr, stream);
}
grid_status grid_fd_f64(const grid_model* m, int N, const double* q, const double* qd,
                        const double* tau, double* qdd, void* stream) {
  grid_status s = check_args<double>(m, N, {q, qd, tau, qdd}, {});
  if (s != GRID_OK) return s;
  return run<double, MODE_FD>(m, N, q, qd, tau, qdd, nullptr, stream);
}
grid_status grid_grad_fd_f64(const grid_model* m, int N, const double* q, const double* qd,
                             const double* tau, double* J, double* qdd, void* stream) {
  grid_status s = check_args<double>(m, N, {q, qd, tau, J}, {qdd});
  if (s != GRID_OK) return s;
  return run<double, MODE_GRAD>(m, N, q, qd, tau, J, qdd, stream);
}

}  // extern "C"
