// D2Q37 instantiations of the fused step, BF16 and FP16 storage (FP32 arithmetic).
#include "step_tma.cuh"

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

// Plain step kernel with diffuse-scattering walls.
void* find_launcher_q37_half_ds(int storage, int coll) {
    switch (storage * 2 + coll) {
        case ST_BF16 * 2 + COLL_BGK:
            return (void*)&launch_step<D2Q37, __nv_bfloat16, COLL_BGK, 1>;
        case ST_BF16 * 2 + COLL_REG:
            return (void*)&launch_step<D2Q37, __nv_bfloat16, COLL_REG, 1>;
        case ST_F16 * 2 + COLL_BGK:
            return (void*)&launch_step<D2Q37, __half, COLL_BGK, 1>;
        case ST_F16 * 2 + COLL_REG:
            return (void*)&launch_step<D2Q37, __half, COLL_REG, 1>;
        default:
            return nullptr;
    }
}

// Plain step with an occupancy floor (16-bit storage): variant 1 = 6, 2 = 7 blocks of 128 per SM.
void* find_occ_launcher_q37_half(int storage, int coll, int variant) {
    switch ((storage * 2 + coll) * 4 + variant) {
        case (ST_BF16 * 2 + COLL_BGK) * 4 + 1:
            return (void*)&launch_step_occ<D2Q37, __nv_bfloat16, COLL_BGK, 6>;
        case (ST_BF16 * 2 + COLL_BGK) * 4 + 2:
            return (void*)&launch_step_occ<D2Q37, __nv_bfloat16, COLL_BGK, 7>;
        case (ST_BF16 * 2 + COLL_REG) * 4 + 1:
            return (void*)&launch_step_occ<D2Q37, __nv_bfloat16, COLL_REG, 6>;
        case (ST_BF16 * 2 + COLL_REG) * 4 + 2:
            return (void*)&launch_step_occ<D2Q37, __nv_bfloat16, COLL_REG, 7>;
        case (ST_F16 * 2 + COLL_BGK) * 4 + 1:
            return (void*)&launch_step_occ<D2Q37, __half, COLL_BGK, 6>;
        case (ST_F16 * 2 + COLL_BGK) * 4 + 2:
            return (void*)&launch_step_occ<D2Q37, __half, COLL_BGK, 7>;
        case (ST_F16 * 2 + COLL_REG) * 4 + 1:
            return (void*)&launch_step_occ<D2Q37, __half, COLL_REG, 6>;
        case (ST_F16 * 2 + COLL_REG) * 4 + 2:
            return (void*)&launch_step_occ<D2Q37, __half, COLL_REG, 7>;
        default:
            return nullptr;
    }
}

// Launchers of the shared-memory-staged step, by variant (tiles in nodes): 10, 11, 12 = one
// node per thread on 32 x 4, 64 x 2, 64 x 4 tiles; 13, 14 = the same on 64 x 2, 64 x 4 tiles with
// the outputs stored through TMA; 20, 21, 22 = two nodes per thread on 64 x 4,
// 64 x 2, 128 x 2 tiles.
void* find_tma_launcher_q37_half(int storage, int coll, int variant) {
    if (variant < 0 || variant >= 32) return nullptr;
    switch ((storage * 2 + coll) * 32 + variant) {
        case (ST_BF16 * 2 + COLL_BGK) * 32 + 10:
            return (void*)&launch_step_tma1<D2Q37, __nv_bfloat16, COLL_BGK, 32, 4>;
        case (ST_BF16 * 2 + COLL_BGK) * 32 + 11:
            return (void*)&launch_step_tma1<D2Q37, __nv_bfloat16, COLL_BGK, 64, 2>;
        case (ST_BF16 * 2 + COLL_BGK) * 32 + 12:
            return (void*)&launch_step_tma1<D2Q37, __nv_bfloat16, COLL_BGK, 64, 4>;
        case (ST_BF16 * 2 + COLL_BGK) * 32 + 13:
            return (void*)&launch_step_tma1s<D2Q37, __nv_bfloat16, COLL_BGK, 64, 2>;
        case (ST_BF16 * 2 + COLL_BGK) * 32 + 14:
            return (void*)&launch_step_tma1s<D2Q37, __nv_bfloat16, COLL_BGK, 64, 4>;
        case (ST_BF16 * 2 + COLL_BGK) * 32 + 20:
            return (void*)&launch_step_pair<D2Q37, __nv_bfloat16, COLL_BGK, 32, 4>;
        case (ST_BF16 * 2 + COLL_BGK) * 32 + 21:
            return (void*)&launch_step_pair<D2Q37, __nv_bfloat16, COLL_BGK, 32, 2>;
        case (ST_BF16 * 2 + COLL_BGK) * 32 + 22:
            return (void*)&launch_step_pair<D2Q37, __nv_bfloat16, COLL_BGK, 64, 2>;
        case (ST_BF16 * 2 + COLL_REG) * 32 + 10:
            return (void*)&launch_step_tma1<D2Q37, __nv_bfloat16, COLL_REG, 32, 4>;
        case (ST_BF16 * 2 + COLL_REG) * 32 + 11:
            return (void*)&launch_step_tma1<D2Q37, __nv_bfloat16, COLL_REG, 64, 2>;
        case (ST_BF16 * 2 + COLL_REG) * 32 + 12:
            return (void*)&launch_step_tma1<D2Q37, __nv_bfloat16, COLL_REG, 64, 4>;
        case (ST_BF16 * 2 + COLL_REG) * 32 + 13:
            return (void*)&launch_step_tma1s<D2Q37, __nv_bfloat16, COLL_REG, 64, 2>;
        case (ST_BF16 * 2 + COLL_REG) * 32 + 14:
            return (void*)&launch_step_tma1s<D2Q37, __nv_bfloat16, COLL_REG, 64, 4>;
        case (ST_BF16 * 2 + COLL_REG) * 32 + 20:
            return (void*)&launch_step_pair<D2Q37, __nv_bfloat16, COLL_REG, 32, 4>;
        case (ST_BF16 * 2 + COLL_REG) * 32 + 21:
            return (void*)&launch_step_pair<D2Q37, __nv_bfloat16, COLL_REG, 32, 2>;
        case (ST_BF16 * 2 + COLL_REG) * 32 + 22:
            return (void*)&launch_step_pair<D2Q37, __nv_bfloat16, COLL_REG, 64, 2>;
        case (ST_F16 * 2 + COLL_BGK) * 32 + 10:
            return (void*)&launch_step_tma1<D2Q37, __half, COLL_BGK, 32, 4>;
        case (ST_F16 * 2 + COLL_BGK) * 32 + 11:
            return (void*)&launch_step_tma1<D2Q37, __half, COLL_BGK, 64, 2>;
        case (ST_F16 * 2 + COLL_BGK) * 32 + 12:
            return (void*)&launch_step_tma1<D2Q37, __half, COLL_BGK, 64, 4>;
        case (ST_F16 * 2 + COLL_BGK) * 32 + 13:
            return (void*)&launch_step_tma1s<D2Q37, __half, COLL_BGK, 64, 2>;
        case (ST_F16 * 2 + COLL_BGK) * 32 + 14:
            return (void*)&launch_step_tma1s<D2Q37, __half, COLL_BGK, 64, 4>;
        case (ST_F16 * 2 + COLL_BGK) * 32 + 20:
            return (void*)&launch_step_pair<D2Q37, __half, COLL_BGK, 32, 4>;
        case (ST_F16 * 2 + COLL_BGK) * 32 + 21:
            return (void*)&launch_step_pair<D2Q37, __half, COLL_BGK, 32, 2>;
        case (ST_F16 * 2 + COLL_BGK) * 32 + 22:
            return (void*)&launch_step_pair<D2Q37, __half, COLL_BGK, 64, 2>;
        case (ST_F16 * 2 + COLL_REG) * 32 + 10:
            return (void*)&launch_step_tma1<D2Q37, __half, COLL_REG, 32, 4>;
        case (ST_F16 * 2 + COLL_REG) * 32 + 11:
            return (void*)&launch_step_tma1<D2Q37, __half, COLL_REG, 64, 2>;
        case (ST_F16 * 2 + COLL_REG) * 32 + 12:
            return (void*)&launch_step_tma1<D2Q37, __half, COLL_REG, 64, 4>;
        case (ST_F16 * 2 + COLL_REG) * 32 + 13:
            return (void*)&launch_step_tma1s<D2Q37, __half, COLL_REG, 64, 2>;
        case (ST_F16 * 2 + COLL_REG) * 32 + 14:
            return (void*)&launch_step_tma1s<D2Q37, __half, COLL_REG, 64, 4>;
        case (ST_F16 * 2 + COLL_REG) * 32 + 20:
            return (void*)&launch_step_pair<D2Q37, __half, COLL_REG, 32, 4>;
        case (ST_F16 * 2 + COLL_REG) * 32 + 21:
            return (void*)&launch_step_pair<D2Q37, __half, COLL_REG, 32, 2>;
        case (ST_F16 * 2 + COLL_REG) * 32 + 22:
            return (void*)&launch_step_pair<D2Q37, __half, COLL_REG, 64, 2>;
        default:
            return nullptr;
    }
}

// Box of the staged kernels for a storage type and tile width bx: width (elements) and left pad.
void tma_box_q37_half(int storage, int bx, int* bw, int* pad) {
    switch (storage) {
        case ST_BF16:
            *pad = TmaGeom<D2Q37, __nv_bfloat16, 2>::PAD;
            *bw = bx + 2 * *pad;
            return;
        case ST_F16:
            *pad = TmaGeom<D2Q37, __half, 2>::PAD;
            *bw = bx + 2 * *pad;
            return;
        default:
            *bw = *pad = 0;
    }
}

}  // namespace lbm
