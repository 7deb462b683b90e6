// Kernel instantiations: double.
#include "grid_launch.cuh"

GRID_INSTANTIATE(double, false)
