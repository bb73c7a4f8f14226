// FP64 squared matrix elements and helicity filter for process 4 (see gen/proc4.cuh).
#include "sigmakin_launch.cuh"
MG_INSTANTIATE_FP64(4)
