// FP32 instantiation of the stencil kernels (FMA contraction on).
#define PPML_REAL float
#include "ppml_kern_impl.cuh"
