// D2Q37 step kernels, FP64 storage and arithmetic (plain kernels only).
#include "step_q37_inst.cuh"

LBM_Q37_EXPORTS(f64, double, false)
