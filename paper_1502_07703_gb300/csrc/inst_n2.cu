// Stage kernels for degree N = 2.
#include "inst.cuh"
PYRDG_INSTANTIATE(2)
