// Kernel-split variant, FP64 kernels, process 4 (see gen/proc4.cuh).
#include "sigmakin_split.cuh"
MG_INSTANTIATE_SPLIT_FP64(4)
