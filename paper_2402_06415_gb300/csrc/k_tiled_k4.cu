// Tiled sweep kernels instantiated for 4 sweeps per launch.
#include "k_tiled.cuh"

ISING_TILED_INSTANTIATE(4)
