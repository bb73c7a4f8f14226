// Squared matrix elements for process 2 (see gen/proc2.cuh).
#include "sigmakin_launch.cuh"
MG_DEFINE_PROCESS_LAUNCHERS(2)
