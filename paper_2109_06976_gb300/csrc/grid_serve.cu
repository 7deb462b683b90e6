// Serving: a persistent kernel that computes the gradient of forward dynamics
// for a stream of MPC requests (mixed robots and horizons), with continuous
// batching across requests, and the native host runtime that feeds it.
//
// Requests live in a ring of slots in mapped pinned host memory; their states
// and Jacobians live in a pinned I/O arena that the GPU reads and writes
// directly over NVLink-C2C (no per-request copies). A request is admitted when
// its ring slot is free and its I/O fits in the arena (first-fit allocation).
// Publishing a request appends its tiles (2 knot points each) to a global unit
// sequence; every warp of the persistent kernel claims the next unit with one
// atomic, so tiles of different requests and robots run side by side as soon
// as they are published. The warp that finishes a request's last tile sets the
// request's done flag with a system-scope release store. Every wait in the
// kernel is bounded by %globaltimer: with no new unit for `idle_ns` the kernel
// records GRID_E_TIMEOUT and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "grid_internal.h"
#include "grid_phases.cuh"

namespace {

constexpr int kServeT = 16;               // lanes per knot point
constexpr int kServeG = 32 / kServeT;     // knot points per tile (one warp)
constexpr int kServeCPL = 2;              // M^-1 columns per lane (n <= 32)
constexpr int kMaxModels = 16;
constexpr int kMaxWarps = 4;

struct ServeReq {                         // one ring slot (host writes, GPU reads)
  unsigned long long q, qd, tau, J;      // device-accessible addresses in the I/O arena
  int model, H, first_unit, nunits;
  int seq;                                // request sequence number; -1 while being written
  int pad[3];
};

struct ServeCtl {                         // control block in mapped pinned memory
  int published_units;                    // host: units made available
  int stop;                               // host: ask the kernel to exit
  int status;                             // GPU: GRID_OK or GRID_E_TIMEOUT
  int pad;
};

__device__ __forceinline__ int ld_acquire_sys(const int* p) {
  int v;
  asm volatile("ld.acquire.sys.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(int* p, int v) {
  asm volatile("st.release.sys.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__host__ __device__ constexpr int align16s(int x) { return (x + 15) & ~15; }

struct ServeArgs {
  const ModelDev<float>* models[kMaxModels];
  int nmodels;
  int ring;                               // slots
  int sched_words;                        // per-warp schedule buffer (uint32)
  int ws_stride;                          // per-warp workspace (floats)
  ServeReq* reqs;                         // [ring], mapped
  ServeCtl* ctl;                          // mapped
  int* done;                              // [ring], mapped: seq of the last finished request
  int* next_unit;                         // device
  int* tiles_done;                        // [ring], device
  unsigned long long idle_ns;
};

// Per-warp shared memory: model head | schedule slice | workspace (2 knot points).
__global__ void __launch_bounds__(32 * kMaxWarps) grid_serve_kernel(ServeArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int head = align16s(model_head_bytes<float>());
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t per_warp = head + align16s(a.sched_words * 4) + (size_t)a.ws_stride * 4;
  unsigned char* base = smem + warp * per_warp;
  ModelDev<float>& M = *reinterpret_cast<ModelDev<float>*>(base);
  uint32_t* sched = reinterpret_cast<uint32_t*>(base + head);
  float* W = reinterpret_cast<float*>(base + head + align16s(a.sched_words * 4));
  int cur_model = -1, nsteps = 0, cursor = 0;
  while (true) {
    int u = 0;
    if (lane == 0) u = atomicAdd(a.next_unit, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    // wait (bounded) until unit u is published
    int ok = 1;
    if (lane == 0) {
      const unsigned long long t0 = globaltimer();
      unsigned ns = 64;
      while (ld_acquire_sys(&a.ctl->published_units) <= u) {
        if (ld_acquire_sys(&a.ctl->stop)) { ok = 0; break; }
        if (globaltimer() - t0 > a.idle_ns) {
          atomicCAS(&a.ctl->status, GRID_OK, GRID_E_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(ns);
        if (ns < 4096) ns *= 2;
      }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return;
    // find the request holding unit u (requests cover increasing unit ranges)
    int slot = 0;
    ServeReq r;
    if (lane == 0) {
      int guard = 0;
      while (true) {
        slot = cursor % a.ring;
        const ServeReq* e = a.reqs + slot;
        const int s1 = ld_acquire_sys(&e->seq);
        r = *e;
        const int s2 = ld_acquire_sys(&e->seq);
        if (s1 == cursor && s2 == cursor && u >= r.first_unit && u < r.first_unit + r.nunits) break;
        if (s1 == cursor && s2 == cursor && u < r.first_unit) { ok = 0; break; }   // inconsistent ring
        ++cursor;                          // request done (slot reused) or u lies further on
        if (++guard > (1 << 24)) { ok = 0; break; }
      }
      if (!ok) atomicCAS(&a.ctl->status, GRID_OK, GRID_E_TIMEOUT);
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return;
    slot = __shfl_sync(0xffffffffu, slot, 0);
    int mi = __shfl_sync(0xffffffffu, r.model, 0);
    const int H = __shfl_sync(0xffffffffu, r.H, 0);
    const int first = __shfl_sync(0xffffffffu, r.first_unit, 0);
    const int nunits = __shfl_sync(0xffffffffu, r.nunits, 0);
    const float* q = reinterpret_cast<const float*>(__shfl_sync(0xffffffffu, r.q, 0));
    const float* qd = reinterpret_cast<const float*>(__shfl_sync(0xffffffffu, r.qd, 0));
    const float* tau = reinterpret_cast<const float*>(__shfl_sync(0xffffffffu, r.tau, 0));
    float* J = reinterpret_cast<float*>(__shfl_sync(0xffffffffu, r.J, 0));
    if (mi != cur_model) {                 // stage this robot's model and schedule slice
      const int4* src = reinterpret_cast<const int4*>(a.models[mi]);
      int4* dst = reinterpret_cast<int4*>(&M);
      for (int i = lane; i < head / 16; i += 32) dst[i] = src[i];
      __syncwarp();
      nsteps = M.steps[1];
      for (int i = lane; i < nsteps * kServeT; i += 32) sched[i] = a.models[mi]->sched[M.sched_off[1] + i];
      __syncwarp();
      cur_model = mi;
    }
    const int k0 = (u - first) * kServeG;
    if (M.maxd > 8)
      process_tile<float, MODE_GRAD, kServeT, kServeCPL, 32, false>(M, a.models[mi], sched, nsteps, W, lane,
                                                                  k0, H, q, qd, tau, nullptr, J, nullptr,
                                                                  nullptr);
    else
      process_tile<float, MODE_GRAD, kServeT, kServeCPL, 8, false>(M, a.models[mi], sched, nsteps, W, lane,
                                                                 k0, H, q, qd, tau, nullptr, J, nullptr,
                                                                 nullptr);
    __threadfence_system();                // this tile's Jacobians are visible to the host
    __syncwarp();
    if (lane == 0) {
      const int old = atomicAdd(a.tiles_done + slot, 1);
      if (old == nunits - 1) {
        a.tiles_done[slot] = 0;
        __threadfence_system();
        st_release_sys(a.done + slot, cursor);
      }
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- host runtime
struct grid_server {
  int device = 0;
  int nmodels = 0;
  int ring = 0;
  const grid_model* models[kMaxModels];
  ServeArgs args{};
  ServeReq* reqs = nullptr;               // mapped pinned (host view)
  ServeCtl* ctl = nullptr;
  int* done = nullptr;
  unsigned char* arena = nullptr;          // mapped pinned I/O arena (host view)
  unsigned char* arena_dev = nullptr;      // its device address
  size_t arena_bytes = 0;
  std::map<size_t, size_t> free_list;      // offset -> bytes
  std::vector<size_t> slot_off, slot_bytes;
  std::vector<int> slot_busy;
  int next_seq = 0;
  int units = 0;
  std::mutex mu;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool running = false;
  size_t smem = 0;
  int grid = 0, threads = 0;
};

namespace {

bool arena_alloc(grid_server* s, size_t bytes, size_t* off) {
  for (auto it = s->free_list.begin(); it != s->free_list.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t noff = it->first + bytes;
      s->free_list.erase(it);
      if (rest) s->free_list[noff] = rest;
      return true;
    }
  }
  return false;
}

void arena_free(grid_server* s, size_t off, size_t bytes) {
  auto it = s->free_list.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != s->free_list.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->free_list.erase(nx);
  }
  if (it != s->free_list.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->free_list.erase(it);
    }
  }
}

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

template <class T>
T load_acq(const T* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
template <class T>
void store_rel(T* p, T v) { __atomic_store_n(p, v, __ATOMIC_RELEASE); }

}  // namespace

extern "C" {

grid_status grid_server_create(const grid_model* const* models, int nmodels, int ring_slots,
                               size_t arena_bytes, grid_server** out) {
  if (!out || !models || nmodels < 1 || nmodels > kMaxModels || ring_slots < 1 || arena_bytes < 4096) {
    grid_set_error("grid_server_create: bad arguments");
    return GRID_E_ARG;
  }
  *out = nullptr;
  grid_server* s = new grid_server();
  cudaGetDevice(&s->device);
  s->nmodels = nmodels;
  s->ring = ring_slots;
  int max_stride = 0, max_sched = 0;
  for (int i = 0; i < nmodels; ++i) {
    if (!models[i] || models[i]->device != s->device) {
      grid_set_error("grid_server_create: model %d missing or on another device", i);
      delete s;
      return GRID_E_ARG;
    }
    if (models[i]->prec != GRID_FP32) {    // the serving kernel has no FP64 pivots
      grid_set_error("grid_server_create: model %d is not an FP32 model (serving runs in FP32)", i);
      delete s;
      return GRID_E_ARG;
    }
    s->models[i] = models[i];
    s->args.models[i] = models[i]->dev_f;
    max_stride = std::max(max_stride, models[i]->host_f->L.stride);
    max_sched = std::max(max_sched, models[i]->host_f->steps[1] * kServeT);
  }
  s->args.nmodels = nmodels;
  s->args.ring = ring_slots;
  s->args.sched_words = max_sched;
  s->args.ws_stride = kServeG * max_stride;
  s->args.idle_ns = 2000000000ull;
  cudaError_t e = cudaHostAlloc(&s->reqs, sizeof(ServeReq) * ring_slots, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostAlloc(&s->ctl, sizeof(ServeCtl), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostAlloc(&s->done, sizeof(int) * ring_slots, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostAlloc(&s->arena, arena_bytes, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaMalloc(&s->args.next_unit, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&s->args.tiles_done, sizeof(int) * ring_slots);
  if (e != cudaSuccess) {
    grid_set_error("grid_server_create: allocation failed: %s", cudaGetErrorString(e));
    cudaFreeHost(s->reqs); cudaFreeHost(s->ctl); cudaFreeHost(s->done); cudaFreeHost(s->arena);
    cudaFree(s->args.next_unit); cudaFree(s->args.tiles_done);
    delete s;
    return GRID_E_NOMEM;
  }
  for (int i = 0; i < ring_slots; ++i) { s->reqs[i].seq = -1; s->done[i] = -1; }
  std::memset(s->ctl, 0, sizeof(ServeCtl));
  cudaHostGetDevicePointer((void**)&s->args.reqs, s->reqs, 0);
  cudaHostGetDevicePointer((void**)&s->args.ctl, s->ctl, 0);
  cudaHostGetDevicePointer((void**)&s->args.done, s->done, 0);
  cudaHostGetDevicePointer((void**)&s->arena_dev, s->arena, 0);
  s->arena_bytes = arena_bytes;
  s->free_list[0] = arena_bytes;
  s->slot_off.assign(ring_slots, 0);
  s->slot_bytes.assign(ring_slots, 0);
  s->slot_busy.assign(ring_slots, 0);
  *out = s;
  return GRID_OK;
}

grid_status grid_server_set_idle_timeout(grid_server* s, double seconds) {
  if (!s || !(seconds > 0)) { grid_set_error("bad idle timeout"); return GRID_E_ARG; }
  if (s->running) { grid_set_error("server already running"); return GRID_E_ARG; }
  s->args.idle_ns = (unsigned long long)(seconds * 1e9);
  return GRID_OK;
}

grid_status grid_server_start(grid_server* s, void* stream) {
  if (!s || s->running) { grid_set_error("grid_server_start: bad server or already running"); return GRID_E_ARG; }
  if (stream) {
    s->stream = reinterpret_cast<cudaStream_t>(stream);
  } else if (!s->own_stream) {
    // a non-blocking stream of its own: the persistent kernel must not hold up
    // (or wait for) work on the legacy default stream
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { grid_set_error("grid_server_start: %s", cudaGetErrorString(e)); return GRID_E_CUDA; }
    s->own_stream = true;
  }
  std::memset(s->ctl, 0, sizeof(ServeCtl));
  s->units = 0;
  cudaMemsetAsync(s->args.next_unit, 0, sizeof(int), s->stream);
  cudaMemsetAsync(s->args.tiles_done, 0, sizeof(int) * s->ring, s->stream);
  const size_t per_warp = align16s(model_head_bytes<float>()) + align16s(s->args.sched_words * 4) +
                          (size_t)s->args.ws_stride * 4;
  int optin = 0, nsm = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
  int warps = kMaxWarps;
  while (warps > 1 && warps * per_warp > (size_t)optin) --warps;
  if (warps * per_warp > (size_t)optin) {
    grid_set_error("grid_server_start: per-warp workspace %zu B exceeds shared memory", per_warp);
    return GRID_E_ARG;
  }
  s->smem = warps * per_warp;
  s->threads = 32 * warps;
  cudaError_t e = cudaFuncSetAttribute(grid_serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e != cudaSuccess) { grid_set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(e)); return GRID_E_CUDA; }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grid_serve_kernel, s->threads, s->smem);
  if (per_sm < 1) { grid_set_error("grid_server_start: kernel does not fit"); return GRID_E_CUDA; }
  s->grid = nsm * per_sm;
  grid_serve_kernel<<<s->grid, s->threads, s->smem, s->stream>>>(s->args);
  e = cudaGetLastError();
  if (e != cudaSuccess) { grid_set_error("grid_server_start: launch: %s", cudaGetErrorString(e)); return GRID_E_CUDA; }
  s->running = true;
  return GRID_OK;
}

grid_status grid_server_submit(grid_server* s, int model, int H, const float* q, const float* qd,
                               const float* tau, long long* request_id) {
  if (!s || !request_id || model < 0 || model >= s->nmodels || H < 1 || !q || !qd || !tau) {
    grid_set_error("grid_server_submit: bad arguments");
    return GRID_E_ARG;
  }
  const int n = s->models[model]->n;
  const size_t in_b = round256(sizeof(float) * H * n);
  const size_t out_b = round256(sizeof(float) * H * 2 * n * n);
  const size_t bytes = 3 * in_b + out_b;
  std::lock_guard<std::mutex> lk(s->mu);
  const int seq = s->next_seq;
  const int slot = seq % s->ring;
  if (s->slot_busy[slot]) { grid_set_error("grid_server_submit: ring slot busy"); return GRID_E_NOMEM; }
  size_t off = 0;
  if (!arena_alloc(s, bytes, &off)) { grid_set_error("grid_server_submit: arena full"); return GRID_E_NOMEM; }
  unsigned char* h = s->arena + off;
  std::memcpy(h, q, sizeof(float) * H * n);
  std::memcpy(h + in_b, qd, sizeof(float) * H * n);
  std::memcpy(h + 2 * in_b, tau, sizeof(float) * H * n);
  ServeReq* e = s->reqs + slot;
  store_rel(&e->seq, -1);
  const unsigned long long d = (unsigned long long)(s->arena_dev + off);
  e->q = d; e->qd = d + in_b; e->tau = d + 2 * in_b; e->J = d + 3 * in_b;
  e->model = model;
  e->H = H;
  e->first_unit = s->units;
  e->nunits = (H + kServeG - 1) / kServeG;
  store_rel(&e->seq, seq);
  s->slot_busy[slot] = 1;
  s->slot_off[slot] = off;
  s->slot_bytes[slot] = bytes;
  s->units += e->nunits;
  s->next_seq = seq + 1;
  store_rel(&s->ctl->published_units, s->units);
  *request_id = seq;
  return GRID_OK;
}

// Wait up to wait_us microseconds (0 = just poll) for request `id`; on success
// copy its Jacobians [H][n][2n] to J (NULL to skip) and release its resources.
grid_status grid_server_result(grid_server* s, long long id, float* J, int wait_us) {
  if (!s || id < 0) { grid_set_error("grid_server_result: bad arguments"); return GRID_E_ARG; }
  const int slot = (int)(id % s->ring);
  auto t0 = std::chrono::steady_clock::now();
  while (load_acq(s->done + slot) != (int)id) {
    if (load_acq(&s->ctl->status) != GRID_OK) {
      grid_set_error("grid_server_result: server kernel stopped (status %d)", s->ctl->status);
      return GRID_E_TIMEOUT;
    }
    auto el = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0);
    if (el.count() >= wait_us) { grid_set_error("grid_server_result: not done"); return GRID_E_TIMEOUT; }
    std::this_thread::yield();
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (J) {
    const ServeReq& e = s->reqs[slot];
    const int n = s->models[e.model]->n;
    const size_t in_b = round256(sizeof(float) * e.H * n);
    std::memcpy(J, s->arena + s->slot_off[slot] + 3 * in_b, sizeof(float) * e.H * 2 * n * n);
  }
  arena_free(s, s->slot_off[slot], s->slot_bytes[slot]);
  s->slot_busy[slot] = 0;
  return GRID_OK;
}

// Ask the kernel to exit and wait for it; returns the kernel's status.
grid_status grid_server_stop(grid_server* s) {
  if (!s) return GRID_E_ARG;
  if (!s->running) return GRID_OK;
  store_rel(&s->ctl->stop, 1);
  cudaError_t e = cudaStreamSynchronize(s->stream);
  s->running = false;
  if (e != cudaSuccess) { grid_set_error("grid_server_stop: %s", cudaGetErrorString(e)); return GRID_E_CUDA; }
  const int st = s->ctl->status;
  if (st != GRID_OK) { grid_set_error("server kernel ended with status %d (idle timeout)", st); }
  return (grid_status)st;
}

int grid_server_kernel_status(const grid_server* s) { return s ? load_acq(&s->ctl->status) : GRID_E_ARG; }

grid_status grid_server_destroy(grid_server* s) {
  if (!s) return GRID_OK;
  if (s->running) grid_server_stop(s);
  cudaFreeHost(s->reqs);
  cudaFreeHost(s->ctl);
  cudaFreeHost(s->done);
  cudaFreeHost(s->arena);
  cudaFree(s->args.next_unit);
  cudaFree(s->args.tiles_done);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
  return GRID_OK;
}

// Open-loop Poisson load: arrivals at `rate_hz` for `seconds`, robot uniform
// over the server's models, horizon uniform over `horizons`; request states
// are slices of the per-model pools (pool_knots knot points of q, qd, tau each,
// [3][pool_knots][n]). Latency runs from the scheduled arrival time to the host
// seeing the done flag. stats: [0] completed, [1] knot points, [2] wall seconds,
// [3] p50 ms, [4] p99 ms, [5] p50 ms (H = 128), [6] p99 ms (H = 128),
// [7] max ms, [8] submissions refused for lack of a slot or arena space.
grid_status grid_server_bench(grid_server* s, double rate_hz, double seconds, unsigned long long seed,
                              const int* horizons, int nh, const float* const* pools, int pool_knots,
                              double* stats) {
  if (!s || !s->running || !(rate_hz > 0) || !(seconds > 0) || !horizons || nh < 1 || !pools || !stats) {
    grid_set_error("grid_server_bench: bad arguments or server not started");
    return GRID_E_ARG;
  }
  for (int i = 0; i < nh; ++i)
    if (horizons[i] < 1 || horizons[i] > pool_knots) { grid_set_error("horizon exceeds pool"); return GRID_E_ARG; }
  // splitmix64 stream for arrivals and choices
  unsigned long long st = seed;
  auto next = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    unsigned long long z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto unit = [&]() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); };
  struct Plan { double t; int model, H, start; };
  std::vector<Plan> plan;
  double t = 0;
  while (true) {
    t += -std::log(1.0 - unit()) / rate_hz;
    if (t >= seconds) break;
    Plan p;
    p.t = t;
    p.model = (int)(unit() * s->nmodels);
    p.H = horizons[(int)(unit() * nh)];
    p.start = (int)(unit() * (pool_knots - p.H + 1));
    plan.push_back(p);
  }
  struct Rec { long long id; double sched; double done; int H; };
  std::vector<Rec> recs(plan.size());
  std::atomic<long long> submitted{0};
  std::atomic<bool> producer_done{false};
  long long refused = 0;
  const auto T0 = std::chrono::steady_clock::now();
  auto now_s = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - T0).count(); };
  std::thread consumer([&]() {
    std::vector<long long> open;            // submitted, not yet seen done
    long long taken = 0;
    while (true) {
      const long long sub = submitted.load(std::memory_order_acquire);
      while (taken < sub) open.push_back(taken++);
      for (size_t i = 0; i < open.size();) {
        Rec& r = recs[open[i]];
        if (grid_server_result(s, r.id, nullptr, 0) == GRID_OK) {
          r.done = now_s();
          open[i] = open.back();
          open.pop_back();
        } else {
          ++i;
        }
      }
      if (open.empty() && producer_done.load() && taken >= submitted.load()) break;
      if (load_acq(&s->ctl->status) != GRID_OK) break;
    }
  });
  for (size_t i = 0; i < plan.size(); ++i) {
    const Plan& p = plan[i];
    while (now_s() < p.t) { }
    const int n = s->models[p.model]->n;
    const float* pool = pools[p.model];
    const float* q = pool + (size_t)p.start * n;
    const float* qd = pool + (size_t)(pool_knots + p.start) * n;
    const float* tau = pool + (size_t)(2 * pool_knots + p.start) * n;
    long long id = -1;
    while (grid_server_submit(s, p.model, p.H, q, qd, tau, &id) != GRID_OK) {
      ++refused;
      std::this_thread::yield();
      if (load_acq(&s->ctl->status) != GRID_OK) break;
    }
    recs[i].id = id;
    recs[i].sched = p.t;
    recs[i].done = -1;
    recs[i].H = p.H;
    submitted.store((long long)i + 1, std::memory_order_release);
  }
  producer_done.store(true);
  consumer.join();
  const double wall = now_s();
  std::vector<double> lat, lat128;
  double knots = 0;
  for (const Rec& r : recs) {
    if (r.done < 0) continue;
    lat.push_back((r.done - r.sched) * 1e3);
    if (r.H == 128) lat128.push_back((r.done - r.sched) * 1e3);
    knots += r.H;
  }
  auto pct = [](std::vector<double> v, double p) {
    if (v.empty()) return -1.0;
    std::sort(v.begin(), v.end());
    const size_t k = (size_t)std::min<double>(v.size() - 1, std::floor(p * (v.size() - 1) + 0.5));
    return v[k];
  };
  stats[0] = (double)lat.size();
  stats[1] = knots;
  stats[2] = wall;
  stats[3] = pct(lat, 0.50);
  stats[4] = pct(lat, 0.99);
  stats[5] = pct(lat128, 0.50);
  stats[6] = pct(lat128, 0.99);
  stats[7] = lat.empty() ? -1.0 : *std::max_element(lat.begin(), lat.end());
  stats[8] = (double)refused;
  if (lat.size() != recs.size()) {
    grid_set_error("grid_server_bench: %zu of %zu requests completed", lat.size(), recs.size());
    return GRID_E_TIMEOUT;
  }
  return GRID_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free batch entry point
// Some callers may not allocate device memory once they are running: a
// real-time control loop that must not call cudaMalloc (it can synchronise the
// device and take unbounded time), or a host application that owns every byte
// of the device and hands the library only its input and output buffers. For
// them grid_serve_batch_static runs a fixed list of requests through the same
// serving kernel in one-shot form, keeping the kernel's scratch (request
// descriptors, control block, done flags and tile counters) in the fixed
// file-scope array below instead of memory allocated per server.
namespace {

constexpr int kStaticMaxReq = 256;        // requests per call (the array's limit)

struct StaticScratch {
  ServeReq reqs[kStaticMaxReq];
  ServeCtl ctl;
  int done[kStaticMaxReq];
  int next_unit;
  int tiles_done[kStaticMaxReq];
};

// Lives on every device that loads this library until the process exits
// (about 18.5 KB). In host code the name is only a stand-in for the symbol;
// its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[sizeof(StaticScratch)];

std::mutex g_static_mu;
void* g_static_addr[64] = {nullptr};      // per device, filled by the first call on it

// The request list travels to the device as a kernel argument (by value, about
// 12 KB), so the call reads no host memory after it returns.
struct StaticList {
  unsigned long long q[kStaticMaxReq], qd[kStaticMaxReq], tau[kStaticMaxReq], J[kStaticMaxReq];
  int model[kStaticMaxReq], H[kStaticMaxReq], first_unit[kStaticMaxReq], nunits[kStaticMaxReq];
  int nreq, units;
};

// Writes the call's descriptors into the scratch array and resets its control
// block, done flags and counters (the previous call's contents are overwritten).
__global__ void static_setup_kernel(StaticScratch* d, const StaticList L) {
  for (int i = threadIdx.x; i < kStaticMaxReq; i += blockDim.x) {
    ServeReq r{};
    const bool live = i < L.nreq;
    r.q = live ? L.q[i] : 0ull;
    r.qd = live ? L.qd[i] : 0ull;
    r.tau = live ? L.tau[i] : 0ull;
    r.J = live ? L.J[i] : 0ull;
    r.model = live ? L.model[i] : 0;
    r.H = live ? L.H[i] : 0;
    r.first_unit = live ? L.first_unit[i] : 0;
    r.nunits = live ? L.nunits[i] : 0;
    r.seq = live ? i : -1;
    d->reqs[i] = r;
    d->done[i] = -1;
    d->tiles_done[i] = 0;
  }
  if (threadIdx.x == 0) {
    d->ctl.published_units = L.units;     // everything is published up front ...
    d->ctl.stop = 1;                      // ... and warps leave once the units run out
    d->ctl.status = GRID_OK;
    d->ctl.pad = 0;
    d->next_unit = 0;
  }
}

}  // namespace

extern "C" grid_status grid_serve_batch_static(const grid_model* const* models, int nmodels, int nreq,
                                               const int* req_model, const int* req_H,
                                               const float* const* q, const float* const* qd,
                                               const float* const* tau, float* const* J, void* stream) {
  if (!models || nmodels < 1 || nmodels > kMaxModels || !req_model || !req_H || !q || !qd || !tau || !J) {
    grid_set_error("grid_serve_batch_static: null or bad argument");
    return GRID_E_ARG;
  }
  if (nreq < 1 || nreq > kStaticMaxReq) {
    grid_set_error("grid_serve_batch_static: %d requests; one call takes 1 to %d", nreq, kStaticMaxReq);
    return GRID_E_ARG;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    grid_set_error("grid_serve_batch_static: no current device");
    return GRID_E_CUDA;
  }
  ServeArgs a{};
  int max_stride = 0, max_sched = 0;
  for (int i = 0; i < nmodels; ++i) {
    if (!models[i] || models[i]->device != dev) {
      grid_set_error("grid_serve_batch_static: model %d missing or on another device", i);
      return GRID_E_ARG;
    }
    if (models[i]->prec != GRID_FP32) {
      grid_set_error("grid_serve_batch_static: model %d is not an FP32 model (serving runs in FP32)", i);
      return GRID_E_ARG;
    }
    a.models[i] = models[i]->dev_f;
    max_stride = std::max(max_stride, models[i]->host_f->L.stride);
    max_sched = std::max(max_sched, models[i]->host_f->steps[1] * kServeT);
  }
  // Set-up once per device, with that device current: the array's device address.
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
      e = cudaGetSymbolAddress(&g_static_addr[dev], g_static_scratch);
      if (e != cudaSuccess) {
        g_static_addr[dev] = nullptr;
        grid_set_error("grid_serve_batch_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return GRID_E_CUDA;
      }
    }
    base = g_static_addr[dev];
  }
  // The request list, passed by value to the set-up kernel on `stream`.
  StaticList L;
  std::memset(&L, 0, sizeof(L));
  int units = 0;
  for (int i = 0; i < nreq; ++i) {
    const int m = req_model[i];
    if (m < 0 || m >= nmodels || req_H[i] < 1 || !q[i] || !qd[i] || !tau[i] || !J[i] ||
        ((uintptr_t)q[i] | (uintptr_t)qd[i] | (uintptr_t)tau[i] | (uintptr_t)J[i]) % sizeof(float)) {
      grid_set_error("grid_serve_batch_static: request %d has a bad model, horizon or pointer", i);
      return GRID_E_ARG;
    }
    L.q[i] = (unsigned long long)q[i];
    L.qd[i] = (unsigned long long)qd[i];
    L.tau[i] = (unsigned long long)tau[i];
    L.J[i] = (unsigned long long)J[i];
    L.model[i] = m;
    L.H[i] = req_H[i];
    L.first_unit[i] = units;
    L.nunits[i] = (req_H[i] + kServeG - 1) / kServeG;
    units += L.nunits[i];
  }
  L.nreq = nreq;
  L.units = units;
  StaticScratch* d = reinterpret_cast<StaticScratch*>(base);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  static_setup_kernel<<<1, 256, 0, st>>>(d, L);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    grid_set_error("grid_serve_batch_static: set-up launch: %s", cudaGetErrorString(e));
    return GRID_E_CUDA;
  }
  a.nmodels = nmodels;
  a.ring = nreq;
  a.sched_words = max_sched;
  a.ws_stride = kServeG * max_stride;
  a.reqs = d->reqs;
  a.ctl = &d->ctl;
  a.done = d->done;
  a.next_unit = &d->next_unit;
  a.tiles_done = d->tiles_done;
  a.idle_ns = 1000000000ull;
  const size_t per_warp = align16s(model_head_bytes<float>()) + align16s(a.sched_words * 4) +
                          (size_t)a.ws_stride * 4;
  int optin = 0, nsm = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int warps = kMaxWarps;
  while (warps > 1 && warps * per_warp > (size_t)optin) --warps;
  if (warps * per_warp > (size_t)optin) {
    grid_set_error("grid_serve_batch_static: per-warp workspace %zu B exceeds shared memory", per_warp);
    return GRID_E_ARG;
  }
  e = cudaFuncSetAttribute(grid_serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e != cudaSuccess) {
    grid_set_error("grid_serve_batch_static: cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    return GRID_E_CUDA;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grid_serve_kernel, 32 * warps, warps * per_warp);
  if (per_sm < 1) {
    grid_set_error("grid_serve_batch_static: kernel does not fit on an SM");
    return GRID_E_CUDA;
  }
  const int blocks = std::min(nsm * per_sm, (units + warps - 1) / warps);
  grid_serve_kernel<<<blocks, 32 * warps, warps * per_warp, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    grid_set_error("grid_serve_batch_static: launch: %s", cudaGetErrorString(e));
    return GRID_E_CUDA;
  }
  return GRID_OK;
}
