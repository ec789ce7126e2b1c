// Stage kernels for degree N = 5.
#include "inst.cuh"
PYRDG_INSTANTIATE(5)
