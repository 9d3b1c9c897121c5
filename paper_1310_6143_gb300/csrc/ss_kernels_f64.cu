// FP64 instantiation: every step in double precision.
#define SS_REAL double
#include "ss_launch.cuh"
