// Kernel-split variant, FP32 kernels and dispatcher, process 1 (see gen/proc1.cuh).
#include "sigmakin_split.cuh"
MG_DEFINE_SPLIT_LAUNCHERS(1)
