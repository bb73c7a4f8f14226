// Squared matrix elements for process 1 (see gen/proc1.cuh).
#include "sigmakin_launch.cuh"
MG_DEFINE_PROCESS_LAUNCHERS(1)
