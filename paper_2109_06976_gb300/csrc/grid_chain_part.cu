// Kernel instantiations for serial chains of 2 .. 8 bodies that are parts of a
// robot (one of its base components, placed in the robot's arrays): as in
// grid_chain.cu, with the placed reads and writes compiled in.
#include "grid_launch.cuh"

template <class S, int MODE>
grid_status launch_chain_part(const grid_model* m, const ModelDev<S>* hm, const ModelDev<S>* dm, int N, const S* q,
                              const S* qd, const S* x3, const S* x4, S* out, S* out2, S* out3, cudaStream_t st) {
  switch (hm->n) {
#define GRID_CHAIN_CASE(NB) \
    case NB: return launch_t<S, MODE, 8, 1, 8, false, 100 + NB>(m, hm, dm, N, q, qd, x3, x4, out, out2, out3, st);
    GRID_CHAIN_CASE(2) GRID_CHAIN_CASE(3) GRID_CHAIN_CASE(4) GRID_CHAIN_CASE(5)
    GRID_CHAIN_CASE(6) GRID_CHAIN_CASE(7) GRID_CHAIN_CASE(8)
#undef GRID_CHAIN_CASE
    default: break;
  }
  grid_set_error("no chain kernel for a part of %d bodies", hm->n);
  return GRID_E_TOPOLOGY;
}

template grid_status launch_chain_part<float, MODE_GRAD>(const grid_model*, const ModelDev<float>*, const ModelDev<float>*,
                                                    int, const float*, const float*, const float*, const float*,
                                                    float*, float*, float*, cudaStream_t);
template grid_status launch_chain_part<double, MODE_GRAD>(const grid_model*, const ModelDev<double>*,
                                                     const ModelDev<double>*, int, const double*, const double*,
                                                     const double*, const double*, double*, double*, double*,
                                                     cudaStream_t);
