// Tiled sweep kernels instantiated for 6 sweeps per launch.
#include "k_tiled.cuh"

ISING_TILED_INSTANTIATE(6)
