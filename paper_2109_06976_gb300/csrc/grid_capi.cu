// C-ABI entry points of include/grid.h: argument checks, model creation and
// destruction, options, and dispatch to the kernels, which are instantiated
// per precision in grid_f32.cu, grid_mixed.cu and grid_f64.cu (see
// grid_launch.cuh for the launch mapping and grid_phases.cuh for the phases).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <initializer_list>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

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

bool forest_compiled(int k, int l);   // grid_forest.cu

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

// ---------------------------------------------------------------- forest branches
bool nb_moving_equals_bodies(int nb, const int* jtype) {
  if (!jtype) return true;
  for (int i = 0; i < nb; ++i)
    if (jtype[i] != GRID_JOINT_REVOLUTE) return false;
  return true;
}

void free_branches(grid_model* m) {
  cudaFree(m->br_dev_f);
  cudaFree(m->br_dev_d);
  delete[] m->br_host_f;
  delete[] m->br_host_d;
  m->br_dev_f = nullptr; m->br_dev_d = nullptr; m->br_host_f = nullptr; m->br_host_d = nullptr;
  m->branches = 0;
}

// The K chain models of a forest of K chains of L bodies (caller bodies c L ..
// c L + L - 1, parent c L - 1 .. of each, the first on the base). Any failure
// leaves branches = 0: the forest kernel then serves the model.
void build_branches(grid_model* m, const int* parent, const double* axis, const double* X_tree,
                    const double* inertia, const double* gravity) {
  const int K = m->forest_k, L = m->forest_l;
  for (int c = 0; c < K; ++c)
    for (int i = 0; i < L; ++i)
      if (parent[c * L + i] != (i == 0 ? -1 : c * L + i - 1)) return;
  m->br_host_f = new ModelDev<float>[K]();
  m->br_host_d = new ModelDev<double>[K]();
  int par[GRID_MAX_DOF];
  for (int i = 0; i < L; ++i) par[i] = i - 1;
  for (int c = 0; c < K; ++c) {
    if (grid_build_model(L, par, nullptr, axis + 3 * c * L, X_tree + 12 * c * L, inertia + 10 * c * L, gravity,
                         &m->br_host_f[c], &m->br_host_d[c]) != GRID_OK) {
      free_branches(m);
      return;
    }
  }
  if (cudaMalloc(&m->br_dev_f, K * sizeof(ModelDev<float>)) != cudaSuccess ||
      cudaMalloc(&m->br_dev_d, K * sizeof(ModelDev<double>)) != cudaSuccess ||
      cudaMemcpy(m->br_dev_f, m->br_host_f, K * sizeof(ModelDev<float>), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->br_dev_d, m->br_host_d, K * sizeof(ModelDev<double>), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    free_branches(m);
    return;
  }
  m->branches = K;
}

// ---------------------------------------------------------------- parts
// A robot whose base components differ (a humanoid's torso with its arms, and
// its legs) gets one model per component, placed in the robot's arrays
// (ModelDev::ld, gslot, gidx, gmask): the components share nothing through the
// fixed base, so each is a problem of its own. Any failure leaves nparts = 0.
}  // namespace

// Streams and events on which small batches run the parts of a robot at the same
// time: the caller's stream forks into one stream per part and joins them again.
// A lock serialises the fork-join sequences of calls on the same model.
struct grid_part_exec {
  std::mutex mu;
  std::vector<cudaStream_t> st;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
};

grid_status grid_parts_fork(const grid_model* m, cudaStream_t caller, cudaStream_t* streams) {
  grid_part_exec* x = m->pexec;
  x->mu.lock();
  cudaError_t e = cudaEventRecord(x->fork, caller);
  for (int p = 0; e == cudaSuccess && p < m->nparts; ++p) {
    e = cudaStreamWaitEvent(x->st[p], x->fork, 0);
    streams[p] = x->st[p];
  }
  if (e != cudaSuccess) {
    x->mu.unlock();
    grid_set_error("parts: fork: %s", cudaGetErrorString(e));
    return GRID_E_CUDA;
  }
  return GRID_OK;
}

grid_status grid_parts_join(const grid_model* m, cudaStream_t caller) {
  grid_part_exec* x = m->pexec;
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < m->nparts; ++p) {
    cudaError_t e1 = cudaEventRecord(x->join[p], x->st[p]);
    cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(caller, x->join[p], 0) : e1;
    if (e == cudaSuccess) e = e2;
  }
  x->mu.unlock();
  if (e != cudaSuccess) {
    grid_set_error("parts: join: %s", cudaGetErrorString(e));
    return GRID_E_CUDA;
  }
  return GRID_OK;
}

namespace {

void free_part_exec(grid_model* m) {
  grid_part_exec* x = m->pexec;
  if (!x) return;
  for (cudaStream_t s : x->st) if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
  for (cudaEvent_t e : x->join) if (e) cudaEventDestroy(e);
  if (x->fork) cudaEventDestroy(x->fork);
  delete x;
  m->pexec = nullptr;
}

void free_parts(grid_model* m) {
  free_part_exec(m);
  for (int p = 0; p < m->nparts; ++p) {
    cudaFree(m->parts[p].dev_f);
    cudaFree(m->parts[p].dev_d);
    delete m->parts[p].host_f;
    delete m->parts[p].host_d;
  }
  delete[] m->parts;
  m->parts = nullptr;
  m->nparts = 0;
}

template <class S>
void place(ModelDev<S>* P, int ld, const std::vector<int>& idx) {
  P->ld = ld;
  P->gmask = 0u;
  for (int s = 0; s < P->n; ++s) {
    P->gslot[s] = idx[s];
    P->gmask |= 1u << idx[s];
  }
  for (int k = 0; k < P->n; ++k) P->gidx[k] = idx[P->perm[k]];
}

void build_parts(grid_model* m, const int* parent, const int* jtype, const double* axis, const double* X_tree,
                 const double* inertia, const double* gravity) {
  const int n = m->n;
  std::vector<int> root(n);
  std::vector<std::vector<int>> comps;
  for (int i = 0; i < n; ++i) {
    root[i] = parent[i] < 0 ? i : root[parent[i]];
    if (parent[i] < 0) comps.emplace_back();
  }
  if (comps.size() < 2) return;
  std::vector<int> slot_of(n), comp_of(n, -1);
  int nc = 0;
  for (int i = 0; i < n; ++i) {
    if (parent[i] < 0) comp_of[i] = nc++;
    else comp_of[i] = comp_of[root[i]];
    slot_of[i] = (int)comps[comp_of[i]].size();
    comps[comp_of[i]].push_back(i);
  }
  m->parts = new grid_part[comps.size()]();
  for (size_t c = 0; c < comps.size(); ++c) {
    const std::vector<int>& idx = comps[c];
    const int k = (int)idx.size();
    std::vector<int> par(k), jt(k);
    std::vector<double> ax(3 * k), xt(12 * k), in(10 * k);
    for (int s = 0; s < k; ++s) {
      const int b = idx[s];
      par[s] = parent[b] < 0 ? -1 : slot_of[parent[b]];
      jt[s] = jtype ? jtype[b] : GRID_JOINT_REVOLUTE;
      for (int a = 0; a < 3; ++a) ax[3 * s + a] = axis[3 * b + a];
      for (int a = 0; a < 12; ++a) xt[12 * s + a] = X_tree[12 * b + a];
      for (int a = 0; a < 10; ++a) in[10 * s + a] = inertia[10 * b + a];
    }
    grid_part& P = m->parts[c];
    P.n = k;
    P.host_f = new ModelDev<float>();
    P.host_d = new ModelDev<double>();
    m->nparts = (int)c + 1;                   // so that free_parts releases this one too
    if (grid_build_model(k, par.data(), jt.data(), ax.data(), xt.data(), in.data(), gravity, P.host_f,
                         P.host_d) != GRID_OK) {
      free_parts(m);
      return;
    }
    place(P.host_f, n, idx);
    place(P.host_d, n, idx);
    P.chain = !P.host_d->any_prism;
    for (int i = 0; P.chain && i < k; ++i) P.chain = P.host_d->parent[i] == i - 1 && P.host_d->perm[i] == i;
    if (cudaMalloc(&P.dev_f, sizeof(ModelDev<float>)) != cudaSuccess ||
        cudaMalloc(&P.dev_d, sizeof(ModelDev<double>)) != cudaSuccess ||
        cudaMemcpy(P.dev_f, P.host_f, sizeof(ModelDev<float>), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P.dev_d, P.host_d, sizeof(ModelDev<double>), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      free_parts(m);
      return;
    }
  }
  grid_part_exec* x = new grid_part_exec();
  m->pexec = x;
  x->st.assign(m->nparts, nullptr);
  x->join.assign(m->nparts, nullptr);
  bool ok = cudaEventCreateWithFlags(&x->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int p = 0; ok && p < m->nparts; ++p)
    ok = cudaStreamCreateWithFlags(&x->st[p], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&x->join[p], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_parts(m);
  }
}

bool all_moving(int nb, const int* jtype) {
  if (!jtype) return true;
  for (int i = 0; i < nb; ++i)
    if (jtype[i] == GRID_JOINT_FIXED) return false;
  return true;
}

// ---------------------------------------------------------------- host buffers
// grid_grad_fd_host: three staging slots and three streams (copy in, kernel,
// copy out). Chunk c uses slot c mod 3; its copy in waits until the copy out of
// the chunk that used the slot before (free[b]), its kernel waits for its copy
// in (loaded[b]), its copy out for its kernel (computed[b]).
}  // namespace

struct grid_host_pipe {
  std::mutex mu;
  size_t slot_bytes = 0;
  void* slot[3] = {nullptr, nullptr, nullptr};
  cudaStream_t st[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t loaded[3] = {}, computed[3] = {}, freed[3] = {}, start = nullptr, done = nullptr;
};

namespace {

std::mutex g_pipe_create;

void host_pipe_free(grid_host_pipe* p) {
  if (!p) return;
  for (int b = 0; b < 3; ++b) {
    if (p->st[b]) cudaStreamSynchronize(p->st[b]);
  }
  for (int b = 0; b < 3; ++b) {
    cudaFree(p->slot[b]);
    if (p->st[b]) cudaStreamDestroy(p->st[b]);
    if (p->loaded[b]) cudaEventDestroy(p->loaded[b]);
    if (p->computed[b]) cudaEventDestroy(p->computed[b]);
    if (p->freed[b]) cudaEventDestroy(p->freed[b]);
  }
  if (p->start) cudaEventDestroy(p->start);
  if (p->done) cudaEventDestroy(p->done);
  delete p;
}

grid_status cuda_fail(const char* what, cudaError_t e) {
  grid_set_error("grid_grad_fd_host: %s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? GRID_E_NOMEM : GRID_E_CUDA;
}

// The model's pipeline, created on first use (streams and events on the model's device).
grid_status host_pipe_get(grid_model* m, grid_host_pipe** out) {
  std::lock_guard<std::mutex> lk(g_pipe_create);
  if (!m->pipe) {
    grid_host_pipe* p = new grid_host_pipe();
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 3 && e == cudaSuccess; ++b) {
      e = cudaStreamCreateWithFlags(&p->st[b], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->loaded[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->computed[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->freed[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      host_pipe_free(p);
      return cuda_fail("stream or event creation", e);
    }
    m->pipe = p;
  }
  *out = m->pipe;
  return GRID_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

template <class S>
grid_status grad_fd_host(const grid_model* mc, int N, const S* q, const S* qd, const S* tau, S* J, S* qdd,
                         void* stream) {
  grid_status s = check_args<S>(mc, N, {q, qd, tau, J}, {qdd});
  if (s != GRID_OK || N == 0) return s;
  grid_model* m = const_cast<grid_model*>(mc);   // the staging is the model's mutable part
  grid_host_pipe* p = nullptr;
  if ((s = host_pipe_get(m, &p)) != GRID_OK) return s;
  std::lock_guard<std::mutex> lk(p->mu);
  const size_t n = (size_t)m->n;
  const size_t out_per = 2 * n * n;                 // scalars of J per knot point
  size_t chunk = (size_t)m->host_chunk_opt;
  if (chunk == 0) chunk = std::max<size_t>(1024, ((32u << 20) / (out_per * sizeof(S))) / 1024 * 1024);
  chunk = std::min(chunk, (size_t)N);
  // slot layout: q, qd, tau, qdd [chunk][n] and J [chunk][n][2n], each 256-byte aligned
  const size_t vec_b = align256(chunk * n * sizeof(S)), mat_b = align256(chunk * out_per * sizeof(S));
  const size_t need = 4 * vec_b + mat_b;
  cudaError_t e;
  if (need > p->slot_bytes) {
    for (int b = 0; b < 3; ++b) {
      if ((e = cudaStreamSynchronize(p->st[b])) != cudaSuccess) return cuda_fail("synchronise", e);
    }
    for (int b = 0; b < 3; ++b) {
      cudaFree(p->slot[b]);
      p->slot[b] = nullptr;
    }
    p->slot_bytes = 0;
    for (int b = 0; b < 3; ++b)
      if ((e = cudaMalloc(&p->slot[b], need)) != cudaSuccess) {
        for (int c = 0; c < 3; ++c) { cudaFree(p->slot[c]); p->slot[c] = nullptr; }
        return cuda_fail("staging allocation", e);
      }
    p->slot_bytes = need;
  }
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  if ((e = cudaEventRecord(p->start, user)) != cudaSuccess) return cuda_fail("event record", e);
  for (int b = 0; b < 3; ++b) cudaStreamWaitEvent(p->st[b], p->start, 0);
  const cudaMemcpyKind h2d = cudaMemcpyHostToDevice, d2h = cudaMemcpyDeviceToHost;
  for (size_t k0 = 0, c = 0; k0 < (size_t)N; k0 += chunk, ++c) {
    const size_t cn = std::min(chunk, (size_t)N - k0);
    const int b = (int)(c % 3);
    char* base = static_cast<char*>(p->slot[b]);
    S* dq = reinterpret_cast<S*>(base);
    S* dqd = reinterpret_cast<S*>(base + vec_b);
    S* dtau = reinterpret_cast<S*>(base + 2 * vec_b);
    S* dqdd = reinterpret_cast<S*>(base + 3 * vec_b);
    S* dJ = reinterpret_cast<S*>(base + 4 * vec_b);
    const size_t vb = cn * n * sizeof(S);
    cudaStreamWaitEvent(p->st[0], p->freed[b], 0);
    e = cudaMemcpyAsync(dq, q + k0 * n, vb, h2d, p->st[0]);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dqd, qd + k0 * n, vb, h2d, p->st[0]);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dtau, tau + k0 * n, vb, h2d, p->st[0]);
    if (e == cudaSuccess) e = cudaEventRecord(p->loaded[b], p->st[0]);
    if (e != cudaSuccess) { s = cuda_fail("copy in", e); break; }
    cudaStreamWaitEvent(p->st[1], p->loaded[b], 0);
    s = run<S, MODE_GRAD>(m, (int)cn, dq, dqd, dtau, nullptr, dJ, qdd ? dqdd : nullptr, nullptr, p->st[1]);
    if (s != GRID_OK) break;
    if ((e = cudaEventRecord(p->computed[b], p->st[1])) != cudaSuccess) { s = cuda_fail("event record", e); break; }
    cudaStreamWaitEvent(p->st[2], p->computed[b], 0);
    e = cudaMemcpyAsync(J + k0 * out_per, dJ, cn * out_per * sizeof(S), d2h, p->st[2]);
    if (e == cudaSuccess && qdd) e = cudaMemcpyAsync(qdd + k0 * n, dqdd, vb, d2h, p->st[2]);
    if (e == cudaSuccess) e = cudaEventRecord(p->freed[b], p->st[2]);
    if (e != cudaSuccess) { s = cuda_fail("copy out", e); break; }
  }
  if (s != GRID_OK) {                   // leave nothing in flight behind an error
    for (int b = 0; b < 3; ++b) cudaStreamSynchronize(p->st[b]);
    return s;
  }
  // the copy out of the last chunk follows every kernel and every copy in
  if ((e = cudaEventRecord(p->done, p->st[2])) != cudaSuccess) return cuda_fail("event record", e);
  if ((e = cudaStreamWaitEvent(user, p->done, 0)) != cudaSuccess) return cuda_fail("stream wait", e);
  return GRID_OK;
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
  m->pipe = nullptr;
  m->host_chunk_opt = 0;
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
  m->branches = 0;
  m->br_dev_f = nullptr; m->br_dev_d = nullptr; m->br_host_f = nullptr; m->br_host_d = nullptr;
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
  // A forest without fixed bodies (caller body i = joint i) also gets one model
  // per chain, built from the caller's arrays, for the branch kernel; without
  // them the forest runs in its own kernel.
  if (m->forest_k > 1 && nb_moving_equals_bodies(n, jtype) && m->n == n)
    build_branches(m, parent, axis, X_tree, inertia, gravity);
  // Base components that the forest kernels do not cover run as parts.
  m->nparts = 0;
  m->parts = nullptr;
  m->pexec = nullptr;
  if (m->host_d->ncomp >= 2 && !(m->forest_k > 1 && forest_compiled(m->forest_k, m->forest_l)) &&
      all_moving(n, jtype) && m->n == n)
    build_parts(m, parent, jtype, axis, X_tree, inertia, gravity);
  *out = m;
  return GRID_OK;
}

grid_status grid_destroy(grid_model* m) {
  if (!m) return GRID_OK;
  cudaDeviceSynchronize();
  cudaFree(m->dev_f);
  cudaFree(m->dev_d);
  grid_gen_cache_free(m->gen);
  host_pipe_free(m->pipe);
  free_branches(m);
  free_parts(m);
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
    if (value != 0 && value != 1 && value != 8 && value != 16 && value != 32) {
      grid_set_error("lanes must be 0, 1, 8, 16 or 32"); return GRID_E_ARG;
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
  } else if (k == "host_chunk") {
    if (value < 0) { grid_set_error("host_chunk must be >= 0"); return GRID_E_ARG; }
    m->host_chunk_opt = value;
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

grid_status grid_grad_fd_host(const grid_model* m, int N, const float* q, const float* qd, const float* tau,
                              float* J, float* qdd, void* stream) {
  return grad_fd_host<float>(m, N, q, qd, tau, J, qdd, stream);
}
grid_status grid_grad_fd_host_f64(const grid_model* m, int N, const double* q, const double* qd,
                                  const double* tau, double* J, double* qdd, void* stream) {
  return grad_fd_host<double>(m, N, q, qd, tau, J, qdd, stream);
}

}  // extern "C"
