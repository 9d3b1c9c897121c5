// FP32-mixed instantiation, part 3: Monte Carlo and the alternative integrators.
#define SS_REAL float
#define SS_PART 3
#include "ss_launch.cuh"
