// Kernel instantiations: float.
#include "grid_launch.cuh"

GRID_INSTANTIATE(float, false)
