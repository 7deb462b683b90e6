// C-ABI entry points of include/grid.h: argument checks, model creation and
// destruction, options, and dispatch to the kernels, which are instantiated
// per precision in grid_f32.cu, grid_mixed.cu and grid_f64.cu (see
// grid_launch.cuh for the launch mapping and grid_phases.cuh for the phases).
#include <cuda_runtime.h>

#include <cstdint>
#include <initializer_list>
#include <string>
#include <type_traits>

#include "grid_internal.h"

template <class S, int MODE, bool MIXED>
grid_status dispatch(const grid_model* m, int N, const S* q, const S* qd, const S* x3, const S* x4,
                     S* out, S* out2, S* out3, cudaStream_t st);

#define GRID_DECLARE(S, MIXED)                                                                       \
  extern template grid_status dispatch<S, MODE_RNEA, MIXED>(const grid_model*, int, const S*,        \
                                                            const S*, const S*, const S*, S*, S*, S*, cudaStream_t); \
  extern template grid_status dispatch<S, MODE_MINV, MIXED>(const grid_model*, int, const S*,        \
                                                            const S*, const S*, const S*, S*, S*, S*, cudaStream_t); \
  extern template grid_status dispatch<S, MODE_FD, MIXED>(const grid_model*, int, const S*,          \
                                                          const S*, const S*, const S*, S*, S*, S*, cudaStream_t); \
  extern template grid_status dispatch<S, MODE_GRAD, MIXED>(const grid_model*, int, const S*,        \
                                                            const S*, const S*, const S*, S*, S*, S*, cudaStream_t); \
  extern template grid_status dispatch<S, MODE_VJP, MIXED>(const grid_model*, int, const S*,         \
                                                           const S*, const S*, const S*, S*, S*, S*, cudaStream_t); \
  extern template grid_status dispatch<S, MODE_GRAD_ID, MIXED>(const grid_model*, int, const S*,     \
                                                           const S*, const S*, const S*, S*, S*, S*, cudaStream_t);
GRID_DECLARE(float, false)
GRID_DECLARE(float, true)
GRID_DECLARE(double, false)

namespace {

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
grid_status run(const grid_model* m, int N, const S* q, const S* qd, const S* x3, const S* x4, S* out,
                S* out2, S* out3, void* stream) {
  if (N == 0) return GRID_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (std::is_same<S, float>::value && m->prec == GRID_MIXED)
    return dispatch<S, MODE, true>(m, N, q, qd, x3, x4, out, out2, out3, st);
  return dispatch<S, MODE, false>(m, N, q, qd, x3, x4, out, out2, out3, st);
}

}  // namespace

// ---------------------------------------------------------------- C-ABI
extern "C" {

grid_status grid_create(int n, const int* parent, const double* axis, const double* X_tree,
                        const double* inertia, const double* gravity, grid_precision prec,
                        grid_model** out) {
  return grid_create_ex(n, parent, nullptr, axis, X_tree, inertia, gravity, prec, out);
}

grid_status grid_create_ex(int n, const int* parent, const int* jtype, const double* axis,
                           const double* X_tree, const double* inertia, const double* gravity,
                           grid_precision prec, grid_model** out) {
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
  m->specialize_opt = 1;
  m->gen = nullptr;
  m->host_f = new ModelDev<float>();
  m->host_d = new ModelDev<double>();
  grid_status s = grid_build_model(n, parent, jtype, axis, X_tree, inertia, gravity, m->host_f, m->host_d);
  if (s != GRID_OK) { delete m->host_f; delete m->host_d; delete m; return s; }
  m->n = m->host_d->n;                       // moving joints
  // A serial chain of revolute joints in caller order (the depth-first
  // numbering is then the identity) can use the chain-specialised kernels.
  m->chain = !m->host_d->any_prism;
  for (int i = 0; m->chain && i < m->n; ++i)
    m->chain = m->host_d->parent[i] == i - 1 && m->host_d->perm[i] == i;
  // K >= 2 identical chains of L bodies on the base, in caller order
  m->forest_k = m->forest_l = 0;
  if (!m->host_d->any_prism) {
    int L = 1;
    while (L < m->n && m->host_d->parent[L] == L - 1) ++L;
    bool ok = m->n % L == 0 && m->n / L >= 2;
    for (int i = 0; ok && i < m->n; ++i)
      ok = m->host_d->parent[i] == (i % L == 0 ? -1 : i - 1) && m->host_d->perm[i] == i;
    if (ok) { m->forest_k = m->n / L; m->forest_l = L; }
  }
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
  grid_gen_cache_free(m->gen);
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
  } else if (k == "specialize") {
    if (value < 0 || value > 2) { grid_set_error("specialize must be 0, 1 or 2"); return GRID_E_ARG; }
    m->specialize_opt = value;
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
  return run<float, MODE_RNEA>(m, N, q, qd, qdd, nullptr, tau, nullptr, nullptr, stream);
}
grid_status grid_minv(const grid_model* m, int N, const float* q, float* Minv, void* stream) {
  grid_status s = check_args<float>(m, N, {q, Minv}, {});
  if (s != GRID_OK) return s;
  return run<float, MODE_MINV>(m, N, q, nullptr, nullptr, nullptr, Minv, nullptr, nullptr, stream);
}
grid_status grid_fd(const grid_model* m, int N, const float* q, const float* qd, const float* tau,
                    float* qdd, void* stream) {
  grid_status s = check_args<float>(m, N, {q, qd, tau, qdd}, {});
  if (s != GRID_OK) return s;
  return run<float, MODE_FD>(m, N, q, qd, tau, nullptr, qdd, nullptr, nullptr, stream);
}
grid_status grid_grad_fd(const grid_model* m, int N, const float* q, const float* qd, const float* tau,
                         float* J, float* qdd, void* stream) {
  grid_status s = check_args<float>(m, N, {q, qd, tau, J}, {qdd});
  if (s != GRID_OK) return s;
  return run<float, MODE_GRAD>(m, N, q, qd, tau, nullptr, J, qdd, nullptr, stream);
}
grid_status grid_grad_fd_ex(const grid_model* m, int N, const float* q, const float* qd, const float* tau,
                            float* J, float* qdd, float* Minv, void* stream) {
  grid_status s = check_args<float>(m, N, {q, qd, tau, J}, {qdd, Minv});
  if (s != GRID_OK) return s;
  return run<float, MODE_GRAD>(m, N, q, qd, tau, nullptr, J, qdd, Minv, stream);
}
grid_status grid_grad_fd_ex_f64(const grid_model* m, int N, const double* q, const double* qd,
                                const double* tau, double* J, double* qdd, double* Minv, void* stream) {
  grid_status s = check_args<double>(m, N, {q, qd, tau, J}, {qdd, Minv});
  if (s != GRID_OK) return s;
  return run<double, MODE_GRAD>(m, N, q, qd, tau, nullptr, J, qdd, Minv, stream);
}
grid_status grid_rnea_f64(const grid_model* m, int N, const double* q, const double* qd,
                          const double* qdd, double* tau, void* stream) {
  grid_status s = check_args<double>(m, N, {q, qd, tau}, {qdd});
  if (s != GRID_OK) return s;
  return run<double, MODE_RNEA>(m, N, q, qd, qdd, nullptr, tau, nullptr, nullptr, stream);
}
grid_status grid_minv_f64(const grid_model* m, int N, const double* q, double* Minv, void* stream) {
  grid_status s = check_args<double>(m, N, {q, Minv}, {});
  if (s != GRID_OK) return s;
  return run<double, MODE_MINV>(m, N, q, nullptr, nullptr, nullptr, Minv, nullptr, nullptr, stream);
}
grid_status grid_fd_f64(const grid_model* m, int N, const double* q, const double* qd,
                        const double* tau, double* qdd, void* stream) {
  grid_status s = check_args<double>(m, N, {q, qd, tau, qdd}, {});
  if (s != GRID_OK) return s;
  return run<double, MODE_FD>(m, N, q, qd, tau, nullptr, qdd, nullptr, nullptr, stream);
}
grid_status grid_grad_fd_f64(const grid_model* m, int N, const double* q, const double* qd,
                             const double* tau, double* J, double* qdd, void* stream) {
  grid_status s = check_args<double>(m, N, {q, qd, tau, J}, {qdd});
  if (s != GRID_OK) return s;
  return run<double, MODE_GRAD>(m, N, q, qd, tau, nullptr, J, qdd, nullptr, stream);
}

grid_status grid_fd_vjp(const grid_model* m, int N, const float* q, const float* qd, const float* tau,
                        const float* gbar, float* dq, float* dqd, float* dtau, void* stream) {
  grid_status s = check_args<float>(m, N, {q, qd, tau, gbar, dq, dqd, dtau}, {});
  if (s != GRID_OK) return s;
  return run<float, MODE_VJP>(m, N, q, qd, tau, gbar, dq, dqd, dtau, stream);
}
grid_status grid_fd_vjp_f64(const grid_model* m, int N, const double* q, const double* qd,
                            const double* tau, const double* gbar, double* dq, double* dqd,
                            double* dtau, void* stream) {
  grid_status s = check_args<double>(m, N, {q, qd, tau, gbar, dq, dqd, dtau}, {});
  if (s != GRID_OK) return s;
  return run<double, MODE_VJP>(m, N, q, qd, tau, gbar, dq, dqd, dtau, stream);
}

grid_status grid_grad_rnea(const grid_model* m, int N, const float* q, const float* qd, const float* qdd,
                           float* dID, void* stream) {
  grid_status s = check_args<float>(m, N, {q, qd, dID}, {qdd});
  if (s != GRID_OK) return s;
  return run<float, MODE_GRAD_ID>(m, N, q, qd, qdd, nullptr, dID, nullptr, nullptr, stream);
}
grid_status grid_grad_rnea_f64(const grid_model* m, int N, const double* q, const double* qd,
                               const double* qdd, double* dID, void* stream) {
  grid_status s = check_args<double>(m, N, {q, qd, dID}, {qdd});
  if (s != GRID_OK) return s;
  return run<double, MODE_GRAD_ID>(m, N, q, qd, qdd, nullptr, dID, nullptr, nullptr, stream);
}

}  // extern "C"
