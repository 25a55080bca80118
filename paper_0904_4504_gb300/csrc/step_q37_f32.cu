// D2Q37 step kernels, FP32 storage.
#include "step_q37_inst.cuh"

LBM_Q37_EXPORTS(f32, float, true)
