// D2Q37 instantiations of the fused step, FP64 and FP32 storage.
#include "step_kernel.cuh"

namespace lbm {

#define LBM_CASE(ST_ENUM, ST, COLL)                                                            \
    case ST_ENUM * 2 + COLL:                                                                   \
        return batched ? (void*)&batch_kernel<D2Q37, ST, COLL> : (void*)&launch_step<D2Q37, ST, COLL>;

void* find_launcher_q37_wide(int storage, int coll, bool batched) {
    switch (storage * 2 + coll) {
        LBM_CASE(ST_F64, double, COLL_BGK)
        LBM_CASE(ST_F64, double, COLL_REG)
        LBM_CASE(ST_F32, float, COLL_BGK)
        LBM_CASE(ST_F32, float, COLL_REG)
        default:
            return nullptr;
    }
}

}  // namespace lbm
