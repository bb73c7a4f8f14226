// Squared matrix elements for process 4 (see gen/proc4.cuh).
#include "sigmakin_launch.cuh"
MG_DEFINE_PROCESS_LAUNCHERS(4)
