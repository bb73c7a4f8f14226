// Kernel-split variant, FP32 kernels and dispatcher, process 3 (see gen/proc3.cuh).
#include "sigmakin_split.cuh"
MG_DEFINE_SPLIT_LAUNCHERS(3)
