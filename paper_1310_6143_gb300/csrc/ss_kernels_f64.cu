// FP64 instantiation: every step in double precision.  Part 1: the Heun passes.
#define SS_REAL double
#define SS_PART 1
#include "ss_launch.cuh"
