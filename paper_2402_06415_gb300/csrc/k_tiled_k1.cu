// Tiled sweep kernels instantiated for 1 sweep per launch.
#include "k_tiled.cuh"

ISING_TILED_INSTANTIATE(1)
