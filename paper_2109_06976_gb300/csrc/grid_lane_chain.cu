// Gradient of FD with one lane per knot point (grid_lane_chain.cuh), for serial
// chains of 2 .. 8 revolute bodies and chains placed in a larger robot.
#include "grid_lane_chain.cuh"

grid_status launch_lane_chain(const grid_model* m, const ModelDev<float>* hm, int ld, const int* slot, int N,
                              const float* q, const float* qd, const float* tau, float* J, float* qdd,
                              float* Minv, cudaStream_t st) {
  return lc_run<MODE_GRAD>(m, hm, ld, slot, N, q, qd, tau, nullptr, J, qdd, Minv, st);
}
