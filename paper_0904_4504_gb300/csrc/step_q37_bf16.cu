// D2Q37 step kernels, BF16 storage, FP32 arithmetic.
#include "step_q37_inst.cuh"

LBM_Q37_EXPORTS(bf16, __nv_bfloat16, true)
