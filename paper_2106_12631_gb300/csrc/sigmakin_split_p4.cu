// Kernel-split variant, FP32 kernels and dispatcher, process 4 (see gen/proc4.cuh).
#include "sigmakin_split.cuh"
MG_DEFINE_SPLIT_LAUNCHERS(4)
