// Step kernels of the FP32 handles (the kernel sources are in k_step.cu).
#define ESPP_STEP_PRECISION 32
#include "k_step.cu"
