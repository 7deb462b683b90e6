// Kernel instantiations for forests of K identical serial chains of L bodies
// on the fixed base (legs of a quadruped, a biped, a hexapod), gradient of FD
// in FP32 and FP64. When the model holds one model per chain (no fixed bodies),
// the chains run independently in the branch kernel (BranchTopo: 8 lanes per
// chain and knot point, the chain kernel's phases). Otherwise the topology and
// the workspace layout of the whole forest are compile-time constants
// (ForestTopo); 8 lanes per knot point, 32 for small batches.
#include "grid_launch.cuh"

bool forest_compiled(int k, int l) {
  const int code = 100 * k + l;
  return code == 403 || code == 206 || code == 404;
}

template <class S, int MODE>
grid_status launch_forest(const grid_model* m, const ModelDev<S>* hm, const ModelDev<S>* dm, int N, const S* q,
                          const S* qd, const S* x3, const S* x4, S* out, S* out2, S* out3, cudaStream_t st) {
  // With one model per chain: the branch kernel, 8 lanes per chain and knot
  // point (a warp holds 4 / K knot points), N K virtual knot points.
  if (m->branches == m->forest_k && (long)N * m->forest_k <= 0x7fffffffL) {
    const ModelDev<S>* bh;
    const ModelDev<S>* bd;
    if constexpr (std::is_same<S, float>::value) { bh = m->br_host_f; bd = m->br_dev_f; }
    else { bh = m->br_host_d; bd = m->br_dev_d; }
    const int NV = N * m->forest_k;
    switch (100 * m->forest_k + m->forest_l) {
      case 403: return launch_t<S, MODE, 8, 1, 8, false, 3, 4>(m, bh, bd, NV, q, qd, x3, x4, out, out2, out3, st);
      case 206: return launch_t<S, MODE, 8, 1, 8, false, 6, 2>(m, bh, bd, NV, q, qd, x3, x4, out, out2, out3, st);
      case 404: return launch_t<S, MODE, 8, 1, 8, false, 4, 4>(m, bh, bd, NV, q, qd, x3, x4, out, out2, out3, st);
      default: break;
    }
  }
  // 8 lanes per knot point for throughput; a batch of at most two knot points
  // per SM is latency-bound and takes one warp per knot point
  const bool lat = N <= 2 * dev_info(m->device).nsm;
  switch (100 * m->forest_k + m->forest_l) {
#define GRID_FOREST(CODE)                                                                                 \
    case CODE:                                                                                            \
      if (lat) return launch_t<S, MODE, 32, 1, 8, false, -CODE>(m, hm, dm, N, q, qd, x3, x4, out, out2, out3, st); \
      return launch_t<S, MODE, 8, 2, 8, false, -CODE>(m, hm, dm, N, q, qd, x3, x4, out, out2, out3, st);
    GRID_FOREST(403)   // 4 legs x 3 joints (12 bodies)
    GRID_FOREST(206)   // 2 chains x 6 joints (12 bodies)
    GRID_FOREST(404)   // 4 legs x 4 joints (16 bodies)
#undef GRID_FOREST
    default:
      break;
  }
  return GRID_E_TOPOLOGY;
}

template grid_status launch_forest<float, MODE_GRAD>(const grid_model*, const ModelDev<float>*,
                                                     const ModelDev<float>*, int, const float*, const float*,
                                                     const float*, const float*, float*, float*, float*,
                                                     cudaStream_t);
template grid_status launch_forest<double, MODE_GRAD>(const grid_model*, const ModelDev<double>*,
                                                      const ModelDev<double>*, int, const double*, const double*,
                                                      const double*, const double*, double*, double*, double*,
                                                      cudaStream_t);
