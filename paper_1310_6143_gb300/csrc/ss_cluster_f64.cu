// FP64 instantiation, part 4: the cluster step of small single systems.
#define SS_REAL double
#define SS_PART 4
#include "ss_cluster.cuh"
