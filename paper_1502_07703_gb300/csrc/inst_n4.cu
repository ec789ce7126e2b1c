// Stage kernels for degree N = 4.
#include "inst.cuh"
PYRDG_INSTANTIATE(4)
