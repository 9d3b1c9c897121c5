// FP32-mixed instantiation, part 2: the persistent and system-block kernels, the
// demagnetising field.
#define SS_REAL float
#define SS_PART 2
#include "ss_launch.cuh"
