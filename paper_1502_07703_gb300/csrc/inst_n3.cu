// Stage kernels for degree N = 3.
#include "inst.cuh"
PYRDG_INSTANTIATE(3)
