// Kernel-split variant, FP64 kernels, process 3 (see gen/proc3.cuh).
#include "sigmakin_split.cuh"
MG_INSTANTIATE_SPLIT_FP64(3)
