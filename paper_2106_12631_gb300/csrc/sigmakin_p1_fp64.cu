// FP64 squared matrix elements and helicity filter for process 1 (see gen/proc1.cuh).
#include "sigmakin_launch.cuh"
MG_INSTANTIATE_FP64(1)
