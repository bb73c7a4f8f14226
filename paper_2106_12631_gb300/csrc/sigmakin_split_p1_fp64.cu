// Kernel-split variant, FP64 kernels, process 1 (see gen/proc1.cuh).
#include "sigmakin_split.cuh"
MG_INSTANTIATE_SPLIT_FP64(1)
