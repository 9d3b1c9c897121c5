// FP32-mixed instantiation: FP32 storage, field and LLG arithmetic; the thermal transform's
// FP64 values rounded to float, FP64 reductions.  Part 1: the Heun passes.
#define SS_REAL float
#define SS_PART 1
#include "ss_launch.cuh"
