// Step kernels of the FP64 handles (the kernel sources are in k_step.cu).
#define ESPP_STEP_PRECISION 64
#include "k_step.cu"
