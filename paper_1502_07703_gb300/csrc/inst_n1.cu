// Stage kernels for degree N = 1.
#include "inst.cuh"
PYRDG_INSTANTIATE(1)
