// Squared matrix elements for process 3 (see gen/proc3.cuh).
#include "sigmakin_launch.cuh"
MG_DEFINE_PROCESS_LAUNCHERS(3)
