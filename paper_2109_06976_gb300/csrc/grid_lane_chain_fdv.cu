// FD and the vector-Jacobian product through FD with one lane per knot point
// (grid_lane_chain.cuh), for serial chains of 2 .. 8 revolute bodies and chains
// placed in a larger robot.
#include "grid_lane_chain.cuh"

grid_status launch_lane_chain_fd(const grid_model* m, const ModelDev<float>* hm, int ld, const int* slot, int N,
                                 const float* q, const float* qd, const float* tau, float* qdd, cudaStream_t st) {
  return lc_run<MODE_FD>(m, hm, ld, slot, N, q, qd, tau, nullptr, qdd, nullptr, nullptr, st);
}

grid_status launch_lane_chain_vjp(const grid_model* m, const ModelDev<float>* hm, int ld, const int* slot, int N,
                                  const float* q, const float* qd, const float* tau, const float* gbar, float* dq,
                                  float* dqd, float* dtau, cudaStream_t st) {
  return lc_run<MODE_VJP>(m, hm, ld, slot, N, q, qd, tau, gbar, dq, dqd, dtau, st);
}
