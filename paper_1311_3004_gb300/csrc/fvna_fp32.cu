// fvna_fp32.cu -- binary32 perturbation-variable kernels (FMA contraction on).
#include "fvna_launch.h"
#include "fvna_sweeps.cuh"

#define POLICY P32
#define SUFFIX fp32
#define HAS_COMP 1
#include "fvna_precision.inc"
