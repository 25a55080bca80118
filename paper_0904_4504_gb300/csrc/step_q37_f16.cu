// D2Q37 step kernels, FP16 storage, FP32 arithmetic.
#include "step_q37_inst.cuh"

LBM_Q37_EXPORTS(f16, __half, true)
