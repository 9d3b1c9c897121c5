// FP32-mixed instantiation: FP32 storage, field and LLG arithmetic; FP64 Box-Muller
// transform and FP64 reductions.
#define SS_REAL float
#include "ss_launch.cuh"
