// Kernel-split variant, FP64 kernels, process 2 (see gen/proc2.cuh).
#include "sigmakin_split.cuh"
MG_INSTANTIATE_SPLIT_FP64(2)
