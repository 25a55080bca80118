// D2Q9 instantiations of the fused step (all storage types, both collisions).
#include "step_kernel.cuh"

namespace lbm {

#define LBM_CASE(ST_ENUM, ST, COLL)                                                            \
    case ST_ENUM * 2 + COLL:                                                                   \
        return batched ? (void*)&batch_kernel<D2Q9, ST, COLL> : (void*)&launch_step<D2Q9, ST, COLL>;

void* find_launcher_q9(int storage, int coll, bool batched) {
    switch (storage * 2 + coll) {
        LBM_CASE(ST_F64, double, COLL_BGK)
        LBM_CASE(ST_F64, double, COLL_REG)
        LBM_CASE(ST_F32, float, COLL_BGK)
        LBM_CASE(ST_F32, float, COLL_REG)
        LBM_CASE(ST_BF16, __nv_bfloat16, COLL_BGK)
        LBM_CASE(ST_BF16, __nv_bfloat16, COLL_REG)
        LBM_CASE(ST_F16, __half, COLL_BGK)
        LBM_CASE(ST_F16, __half, COLL_REG)
        default:
            return nullptr;
    }
}

}  // namespace lbm
