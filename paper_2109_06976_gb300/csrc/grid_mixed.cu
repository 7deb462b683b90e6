// Kernel instantiations: float with FP64 pivots.
#include "grid_launch.cuh"

GRID_INSTANTIATE(float, true)
