// Stage kernels for degree N = 6.
#include "inst.cuh"
PYRDG_INSTANTIATE(6)
