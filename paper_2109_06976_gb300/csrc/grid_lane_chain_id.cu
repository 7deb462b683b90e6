// RNEA, M^-1 and the gradient of ID with one lane per knot point
// (grid_lane_chain.cuh), for serial chains of 2 .. 8 revolute bodies and chains
// placed in a larger robot.
#include "grid_lane_chain.cuh"

grid_status launch_lane_chain_rnea(const grid_model* m, const ModelDev<float>* hm, int ld, const int* slot, int N,
                                   const float* q, const float* qd, const float* qdd, float* tau, cudaStream_t st) {
  return lc_run<MODE_RNEA>(m, hm, ld, slot, N, q, qd, qdd, nullptr, tau, nullptr, nullptr, st);
}

grid_status launch_lane_chain_minv(const grid_model* m, const ModelDev<float>* hm, int ld, const int* slot, int N,
                                   const float* q, float* Minv, cudaStream_t st) {
  return lc_run<MODE_MINV>(m, hm, ld, slot, N, q, nullptr, nullptr, nullptr, Minv, nullptr, nullptr, st);
}

grid_status launch_lane_chain_grad_id(const grid_model* m, const ModelDev<float>* hm, int ld, const int* slot,
                                      int N, const float* q, const float* qd, const float* qdd, float* D,
                                      cudaStream_t st) {
  return lc_run<MODE_GRAD_ID>(m, hm, ld, slot, N, q, qd, qdd, nullptr, D, nullptr, nullptr, st);
}
