// Kernel-split variant, FP32 kernels and dispatcher, process 2 (see gen/proc2.cuh).
#include "sigmakin_split.cuh"
MG_DEFINE_SPLIT_LAUNCHERS(2)
