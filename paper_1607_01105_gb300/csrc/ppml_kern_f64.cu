// FP64 instantiation of the stencil kernels.  Built with -fmad=false so that every
// expression is evaluated exactly as written (the same order as the FP64 checker).
#define PPML_REAL double
#include "ppml_kern_impl.cuh"
