// D2Q37 instantiations of the in-place (AA) step, BF16 and FP16 storage (FP32 arithmetic).
#include "step_aa.cuh"

namespace lbm {

#define LBM_AA(ST_ENUM, ST, COLL)                                                         \
    case (ST_ENUM * 2 + COLL) * 2 + 0:                                                    \
        return &launch_step_aa<D2Q37, ST, COLL, 0>;                                       \
    case (ST_ENUM * 2 + COLL) * 2 + 1:                                                    \
        return &launch_step_aa<D2Q37, ST, COLL, 1>;

StepLaunchFn find_aa_launcher_q37_half(int storage, int coll, int phase) {
    switch ((storage * 2 + coll) * 2 + phase) {
        LBM_AA(ST_BF16, __nv_bfloat16, COLL_BGK)
        LBM_AA(ST_BF16, __nv_bfloat16, COLL_REG)
        LBM_AA(ST_F16, __half, COLL_BGK)
        LBM_AA(ST_F16, __half, COLL_REG)
        default:
            return nullptr;
    }
}

}  // namespace lbm
