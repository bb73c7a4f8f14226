// FP64 squared matrix elements and helicity filter for process 3 (see gen/proc3.cuh).
#include "sigmakin_launch.cuh"
MG_INSTANTIATE_FP64(3)
