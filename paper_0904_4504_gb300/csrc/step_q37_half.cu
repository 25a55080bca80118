// D2Q37 instantiations of the fused step, BF16 and FP16 storage (FP32 arithmetic).
#include "step_kernel.cuh"

namespace lbm {

#define LBM_CASE(ST_ENUM, ST, COLL)                                                            \
    case ST_ENUM * 2 + COLL:                                                                   \
        return batched ? (void*)&batch_kernel<D2Q37, ST, COLL> : (void*)&launch_step<D2Q37, ST, COLL>;

void* find_launcher_q37_half(int storage, int coll, bool batched) {
    switch (storage * 2 + coll) {
        LBM_CASE(ST_BF16, __nv_bfloat16, COLL_BGK)
        LBM_CASE(ST_BF16, __nv_bfloat16, COLL_REG)
        LBM_CASE(ST_F16, __half, COLL_BGK)
        LBM_CASE(ST_F16, __half, COLL_REG)
        default:
            return nullptr;
    }
}

}  // namespace lbm
