// Stage kernels for degree N = 7.
#include "inst.cuh"
PYRDG_INSTANTIATE(7)
