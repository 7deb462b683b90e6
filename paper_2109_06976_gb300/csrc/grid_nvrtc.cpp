// Run-time specialisation of the gradient-of-FD kernel for one robot's
// topology (grid_set_option "specialize" = 2). The device headers of the
// library (embedded at build time) are compiled by NVRTC together with the
// robot's topology tables as compile-time constants, so that the loops over
// bodies unroll and fold as in the chain and forest kernels, for any tree.
// NVRTC and the CUDA driver are loaded on first use; without them the call
// reports GRID_E_CUDA.
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "grid_internal.h"
#include "grid_embed.inc"   // kEmbedCount, kEmbedNames[], kEmbedSources[] (generated by build_ext.py)

namespace {

struct Api {
  bool ok = false;
  std::string why;
  nvrtcResult (*createProgram)(nvrtcProgram*, const char*, const char*, int, const char* const*,
                               const char* const*) = nullptr;
  nvrtcResult (*compileProgram)(nvrtcProgram, int, const char* const*) = nullptr;
  nvrtcResult (*getProgramLogSize)(nvrtcProgram, size_t*) = nullptr;
  nvrtcResult (*getProgramLog)(nvrtcProgram, char*) = nullptr;
  nvrtcResult (*getCUBINSize)(nvrtcProgram, size_t*) = nullptr;
  nvrtcResult (*getCUBIN)(nvrtcProgram, char*) = nullptr;
  nvrtcResult (*destroyProgram)(nvrtcProgram*) = nullptr;
  CUresult (*moduleLoadData)(CUmodule*, const void*) = nullptr;
  CUresult (*moduleGetFunction)(CUfunction*, CUmodule, const char*) = nullptr;
  CUresult (*funcSetAttribute)(CUfunction, CUfunction_attribute, int) = nullptr;
  CUresult (*occupancy)(int*, CUfunction, int, size_t) = nullptr;
  CUresult (*launchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                           CUstream, void**, void**) = nullptr;
  CUresult (*moduleUnload)(CUmodule) = nullptr;
};

template <class F>
bool sym(void* lib, const char* name, F& f) {
  f = reinterpret_cast<F>(dlsym(lib, name));
  return f != nullptr;
}

const Api& api() {
  static Api a;
  static std::once_flag once;
  std::call_once(once, [] {
    void* nv = dlopen("libnvrtc.so.13", RTLD_NOW | RTLD_LOCAL);
    if (!nv) nv = dlopen("/usr/local/cuda/lib64/libnvrtc.so.13", RTLD_NOW | RTLD_LOCAL);
    void* cu = dlopen("libcuda.so.1", RTLD_NOW | RTLD_LOCAL);
    if (!nv || !cu) {
      a.why = !nv ? "libnvrtc.so.13 not found" : "libcuda.so.1 not found";
      return;
    }
    bool ok = sym(nv, "nvrtcCreateProgram", a.createProgram) && sym(nv, "nvrtcCompileProgram", a.compileProgram) &&
              sym(nv, "nvrtcGetProgramLogSize", a.getProgramLogSize) &&
              sym(nv, "nvrtcGetProgramLog", a.getProgramLog) && sym(nv, "nvrtcGetCUBINSize", a.getCUBINSize) &&
              sym(nv, "nvrtcGetCUBIN", a.getCUBIN) && sym(nv, "nvrtcDestroyProgram", a.destroyProgram) &&
              sym(cu, "cuModuleLoadData", a.moduleLoadData) && sym(cu, "cuModuleGetFunction", a.moduleGetFunction) &&
              sym(cu, "cuFuncSetAttribute", a.funcSetAttribute) &&
              sym(cu, "cuOccupancyMaxActiveBlocksPerMultiprocessor", a.occupancy) &&
              sym(cu, "cuLaunchKernel", a.launchKernel) && sym(cu, "cuModuleUnload", a.moduleUnload);
    a.ok = ok;
    if (!ok) a.why = "missing NVRTC or driver entry point";
  });
  return a;
}

template <class S>
void table(std::string& src, const char* name, const int* v, int n) {
  src += "__device__ constexpr int " + std::string(name) + "[" + std::to_string(n) + "] = {";
  for (int i = 0; i < n; ++i) src += (i ? ", " : "") + std::to_string(v[i]);
  src += "};\n";
}

// The kernel source for one model, scalar type, lane count and accumulator depth.
template <class S>
std::string kernel_source(const ModelDev<S>& D, int T, int CPL, int MAXD) {
  const int n = D.n;
  std::string s = "#include \"grid_kernel.cuh\"\n";
  table<S>(s, "kParent", D.parent, n);
  table<S>(s, "kDepth", D.depth, n);
  table<S>(s, "kSubEnd", D.sub_end, n);
  table<S>(s, "kCompLo", D.comp_lo, n);
  table<S>(s, "kCompHi", D.comp_hi, n);
  table<S>(s, "kPerm", D.perm, n);
  table<S>(s, "kSkoff", D.skoff, n);
  table<S>(s, "kBranch", D.branch, n);
  table<S>(s, "kJt", D.jt, n);
  const std::string N = std::to_string(n);
  s += "template <class S, int MODE>\nstruct GenTopo {\n"
       "  static constexpr int kUnroll = " + N + ";\n"
       "  static constexpr int kChainN = 0;\n"
       "  static constexpr bool kConsecutivePaths = false;\n"
       "  static constexpr int kPlace = 2;\n"
       "  static constexpr int kBranches = 0;\n"
       "  __device__ explicit GenTopo(const ModelDev<S>&) {}\n"
       "  GRID_HD static constexpr KnotLayout layout() { return make_layout(" + N + ", " + std::to_string(D.nsk) +
       ", " + std::to_string(D.nbranch) + ", (int)sizeof(S), layout_kind(MODE)); }\n"
       "  GRID_HD static constexpr int n() { return " + N + "; }\n"
       "  GRID_HD static constexpr int maxd() { return " + std::to_string(D.maxd) + "; }\n"
       "  GRID_HD static constexpr int nbranch() { return " + std::to_string(D.nbranch) + "; }\n"
       "  __device__ static constexpr int parent(int i) { return kParent[i]; }\n"
       "  __device__ static constexpr int depth(int i) { return kDepth[i]; }\n"
       "  __device__ static constexpr int sub_end(int i) { return kSubEnd[i]; }\n"
       "  __device__ static constexpr int comp_lo(int i) { return kCompLo[i]; }\n"
       "  __device__ static constexpr int comp_hi(int i) { return kCompHi[i]; }\n"
       "  __device__ static constexpr int perm(int i) { return kPerm[i]; }\n"
       "  __device__ static constexpr int skoff(int i) { return kSkoff[i]; }\n"
       "  __device__ static constexpr int branch(int i) { return kBranch[i]; }\n"
       "  __device__ static constexpr bool prism(int i) { return kJt[i] != 0; }\n"
       "};\n";
  const std::string Sn = sizeof(S) == 4 ? "float" : "double";
  s += "extern \"C\" __global__ void __launch_bounds__(128) grid_gen_kernel(const ModelDev<" + Sn +
       ">* gm, int N, const " + Sn + "* q, const " + Sn + "* qd, const " + Sn + "* x3, const " + Sn + "* x4, " + Sn +
       "* out, " + Sn + "* out2, " + Sn + "* out3) {\n"
       "  grid_kernel_body<" + Sn + ", MODE_GRAD, " + std::to_string(T) + ", " + std::to_string(CPL) + ", " +
       std::to_string(MAXD) + ", false, GenTopo<" + Sn + ", MODE_GRAD>>(gm, N, q, qd, x3, x4, out, out2, out3);\n}\n";
  return s;
}

}  // namespace

// Compiled kernels of one model, by (scalar size, lanes, columns per lane, depth bound).
struct grid_gen_cache {
  std::mutex mu;
  struct Entry {
    const void* topo;          // the host model whose topology was compiled (the robot, or one of its parts)
    int ssize, T, CPL, MAXD;
    CUmodule mod;
    CUfunction fn;
    int warps, per_sm;
  };
  std::vector<Entry> entries;
};

void grid_gen_cache_free(grid_gen_cache* c) {
  if (!c) return;
  if (api().ok)
    for (auto& e : c->entries) api().moduleUnload(e.mod);
  delete c;
}

template <class S>
grid_status grid_gen_launch(grid_model* m, const ModelDev<S>* hm, const ModelDev<S>* dm, int N, const S* q,
                            const S* qd, const S* tau, S* J, S* qdd, S* Minv, int T, int CPL, int MAXD, int nsm,
                            int smem_optin, cudaStream_t st) {
  const Api& A = api();
  if (!A.ok) {
    grid_set_error("run-time specialisation unavailable: %s", A.why.c_str());
    return GRID_E_CUDA;
  }
  if (!m->gen) m->gen = new grid_gen_cache();
  grid_gen_cache& C = *m->gen;
  grid_gen_cache::Entry* e = nullptr;
  {
    std::lock_guard<std::mutex> lk(C.mu);
    for (auto& x : C.entries)
      if (x.topo == (const void*)hm && x.ssize == (int)sizeof(S) && x.T == T && x.CPL == CPL && x.MAXD == MAXD)
        e = &x;
    if (!e) {
      const std::string src = kernel_source<S>(*hm, T, CPL, MAXD);
      nvrtcProgram prog;
      if (A.createProgram(&prog, src.c_str(), "grid_gen.cu", kEmbedCount, kEmbedSources, kEmbedNames) !=
          NVRTC_SUCCESS) {
        grid_set_error("nvrtcCreateProgram failed");
        return GRID_E_CUDA;
      }
      const std::string hf = "-DGRID_RTC_HEAD_F=" + std::to_string(model_head_bytes<float>());
      const std::string hd = "-DGRID_RTC_HEAD_D=" + std::to_string(model_head_bytes<double>());
      const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device", hf.c_str(), hd.c_str()};
      const nvrtcResult cr = A.compileProgram(prog, 5, opts);
      if (cr != NVRTC_SUCCESS) {
        size_t ls = 0;
        A.getProgramLogSize(prog, &ls);
        std::string log(ls, '\0');
        A.getProgramLog(prog, &log[0]);
        A.destroyProgram(&prog);
        grid_set_error("NVRTC compile failed: %.400s", log.c_str());
        return GRID_E_CUDA;
      }
      size_t cs = 0;
      A.getCUBINSize(prog, &cs);
      std::vector<char> cubin(cs);
      A.getCUBIN(prog, cubin.data());
      A.destroyProgram(&prog);
      grid_gen_cache::Entry x{(const void*)hm, (int)sizeof(S), T, CPL, MAXD, nullptr, nullptr, 0, 0};
      if (A.moduleLoadData(&x.mod, cubin.data()) != CUDA_SUCCESS ||
          A.moduleGetFunction(&x.fn, x.mod, "grid_gen_kernel") != CUDA_SUCCESS ||
          A.funcSetAttribute(x.fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, smem_optin) != CUDA_SUCCESS) {
        grid_set_error("loading the specialised kernel failed");
        return GRID_E_CUDA;
      }
      C.entries.push_back(x);
      e = &C.entries.back();
    }
  }
  const int G = 32 / T;
  const int nsteps = hm->steps[T == 8 ? 0 : (T == 16 ? 1 : 2)];
  const size_t fixed = (size_t)((model_head_bytes<S>() + 15) & ~15) + ((nsteps * T * 4 + 15) & ~15);
  const size_t per_warp = (size_t)G * hm->L.stride * sizeof(S);
  if (!e->warps) {
    int best = 0;
    for (int w = 4; w >= 1; --w) {
      const size_t sm = fixed + w * per_warp;
      if (sm > (size_t)smem_optin) continue;
      int b = 0;
      A.occupancy(&b, e->fn, 32 * w, sm);
      if (b * w > best) { best = b * w; e->warps = w; e->per_sm = b; }
    }
    if (!e->warps) {
      grid_set_error("knot workspace exceeds shared memory; use more lanes");
      return GRID_E_ARG;
    }
  }
  const long tiles = (N + G - 1) / G;
  const unsigned grid = (unsigned)std::min<long>((tiles + e->warps - 1) / e->warps, (long)nsm * e->per_sm);
  const S* x4 = nullptr;
  void* args[] = {(void*)&dm, (void*)&N, (void*)&q, (void*)&qd, (void*)&tau, (void*)&x4, (void*)&J, (void*)&qdd,
                  (void*)&Minv};
  if (A.launchKernel(e->fn, grid, 1, 1, 32 * e->warps, 1, 1, (unsigned)(fixed + e->warps * per_warp),
                     reinterpret_cast<CUstream>(st), args, nullptr) != CUDA_SUCCESS) {
    grid_set_error("launching the specialised kernel failed");
    return GRID_E_CUDA;
  }
  return GRID_OK;
}

template grid_status grid_gen_launch<float>(grid_model*, const ModelDev<float>*, const ModelDev<float>*, int,
                                            const float*, const float*, const float*, float*, float*, float*, int,
                                            int, int, int, int, cudaStream_t);
template grid_status grid_gen_launch<double>(grid_model*, const ModelDev<double>*, const ModelDev<double>*, int,
                                             const double*, const double*, const double*, double*, double*,
                                             double*, int, int, int, int, int, cudaStream_t);
