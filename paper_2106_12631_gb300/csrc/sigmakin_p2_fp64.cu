// FP64 squared matrix elements and helicity filter for process 2 (see gen/proc2.cuh).
#include "sigmakin_launch.cuh"
MG_INSTANTIATE_FP64(2)
