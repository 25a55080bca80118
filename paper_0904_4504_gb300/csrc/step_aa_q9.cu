// D2Q9 instantiations of the in-place (AA) step, every storage type.
#include "step_aa.cuh"

namespace lbm {

#define LBM_AA(ST_ENUM, ST, COLL)                                                         \
    case (ST_ENUM * 2 + COLL) * 2 + 0:                                                    \
        return &launch_step_aa<D2Q9, ST, COLL, 0>;                                        \
    case (ST_ENUM * 2 + COLL) * 2 + 1:                                                    \
        return &launch_step_aa<D2Q9, ST, COLL, 1>;

StepLaunchFn find_aa_launcher_q9(int storage, int coll, int phase) {
    switch ((storage * 2 + coll) * 2 + phase) {
        LBM_AA(ST_F64, double, COLL_BGK)
        LBM_AA(ST_F64, double, COLL_REG)
        LBM_AA(ST_F32, float, COLL_BGK)
        LBM_AA(ST_F32, float, COLL_REG)
        LBM_AA(ST_BF16, __nv_bfloat16, COLL_BGK)
        LBM_AA(ST_BF16, __nv_bfloat16, COLL_REG)
        LBM_AA(ST_F16, __half, COLL_BGK)
        LBM_AA(ST_F16, __half, COLL_REG)
        default:
            return nullptr;
    }
}

}  // namespace lbm
