// fvna_3d32.cu -- the 3D step in binary32 perturbation variables (q1 - 1,
// q2, q3, q4); FMA contraction on.
#include "fvna_3d.cuh"
#include "fvna_launch3.h"

#define T3 float
#define SFX 32
#define HAS_COMP3 1
#include "fvna_3d.inc"
