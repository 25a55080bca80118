// D2Q9 instantiations of the fused step (all storage types, both collisions).
#include "pbatch.cuh"
#include "step_q9v.cuh"

namespace lbm {

#define LBM_CASE(ST_ENUM, ST, COLL)                                                            \
    case ST_ENUM * 2 + COLL:                                                                   \
        return (void*)&launch_step<D2Q9, ST, COLL>;

void* find_launcher_q9(int storage, int coll) {
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

#undef LBM_CASE

// The persistent batch kernel (pbatch.cuh), by the variant whose tile code it runs: 27 = staged
// 64 x 3 tiles (16-bit storage, FP32), 0 = plain 32 x 4 tiles.
template <class ST, int COLL>
PbKernel q9_pbatch_c(int variant) {
    constexpr bool wide = sizeof(ST) == 8;
    if constexpr (!wide) {
        if (variant == 27)
            return pbatch_kernel_info<D2Q9, ST, COLL, PB_STAGED, 64, 3, sizeof(ST) == 2 ? 16 : 12>();
    }
    if (variant == 0) return pbatch_kernel_info<D2Q9, ST, COLL, PB_PLAIN, 32, 4, wide ? 6 : 8>();
    return PbKernel{nullptr, dim3(), 0, 0, 0};
}

template <class ST>
PbKernel q9_pbatch_s(int coll, int variant) {
    if (coll == COLL_REG) return q9_pbatch_c<ST, COLL_REG>(variant);
    if (coll == COLL_BGK) return q9_pbatch_c<ST, COLL_BGK>(variant);
    return PbKernel{nullptr, dim3(), 0, 0, 0};
}

PbKernel find_pbatch_q9(int storage, int coll, int variant) {
    switch (storage) {
        case ST_F64: return q9_pbatch_s<double>(coll, variant);
        case ST_F32: return q9_pbatch_s<float>(coll, variant);
        case ST_BF16: return q9_pbatch_s<__nv_bfloat16>(coll, variant);
        case ST_F16: return q9_pbatch_s<__half>(coll, variant);
        default: return PbKernel{nullptr, dim3(), 0, 0, 0};
    }
}

// The four-nodes-per-thread kernel of 16-bit storage (variant 30, 128 x 4 tiles; step_q9v.cuh).
// The kernel is latency bound, so the occupancy floor is set above what the registers alone
// give: the regularized collision at 8 blocks per SM (64 registers, 8 B spilled; measured 0.62 /
// 0.73 of the copy peak at 2048^2 / 4096^2 against 0.56 / 0.63 at its unspilled 6 blocks, 0.61 /
// 0.72 at 9 and 0.53 / 0.62 at 10), plain BGK at 7 (0.57 against 0.55 at 6 and 8).  (Two rows per
// thread with both rows' loads issued first, 128 x 8 tiles, measured 0.54-0.64 against 0.56-0.63
// on the same box: not built.)
void* find_q9v_launcher(int storage, int coll, int variant) {
    if (variant != 30) return nullptr;
    switch (storage * 2 + coll) {
        case ST_BF16 * 2 + COLL_BGK: return (void*)&launch_step_q9v<__nv_bfloat16, COLL_BGK, 1, 7>;
        case ST_BF16 * 2 + COLL_REG: return (void*)&launch_step_q9v<__nv_bfloat16, COLL_REG, 1, 8>;
        case ST_F16 * 2 + COLL_BGK: return (void*)&launch_step_q9v<__half, COLL_BGK, 1, 7>;
        case ST_F16 * 2 + COLL_REG: return (void*)&launch_step_q9v<__half, COLL_REG, 1, 8>;
        default: return nullptr;
    }
}

// Plain step kernel with diffuse-scattering walls.
void* find_launcher_q9_ds(int storage, int coll) {
    switch (storage * 2 + coll) {
        case ST_F64 * 2 + COLL_BGK:
            return (void*)&launch_step<D2Q9, double, COLL_BGK, 1>;
        case ST_F64 * 2 + COLL_REG:
            return (void*)&launch_step<D2Q9, double, COLL_REG, 1>;
        case ST_F32 * 2 + COLL_BGK:
            return (void*)&launch_step<D2Q9, float, COLL_BGK, 1>;
        case ST_F32 * 2 + COLL_REG:
            return (void*)&launch_step<D2Q9, float, COLL_REG, 1>;
        case ST_BF16 * 2 + COLL_BGK:
            return (void*)&launch_step<D2Q9, __nv_bfloat16, COLL_BGK, 1>;
        case ST_BF16 * 2 + COLL_REG:
            return (void*)&launch_step<D2Q9, __nv_bfloat16, COLL_REG, 1>;
        case ST_F16 * 2 + COLL_BGK:
            return (void*)&launch_step<D2Q9, __half, COLL_BGK, 1>;
        case ST_F16 * 2 + COLL_REG:
            return (void*)&launch_step<D2Q9, __half, COLL_REG, 1>;
        default:
            return nullptr;
    }
}

// Launchers of the shared-memory-staged step, by variant (tiles in nodes): 10 = one node per
// thread on 32 x 4 tiles; 20 = two nodes per thread on 64 x 4 tiles; 27 = 64 x 1 threads, three
// rows each (64 x 3 tiles, the persistent batch kernel's staged shape).
void* find_tma_launcher_q9(int storage, int coll, int variant) {
    if (variant < 0 || variant >= 32) return nullptr;
    switch ((storage * 2 + coll) * 32 + variant) {
        case (ST_F32 * 2 + COLL_BGK) * 32 + 10:
            return (void*)&launch_step_tma1<D2Q9, float, COLL_BGK, 32, 4>;
        case (ST_F32 * 2 + COLL_BGK) * 32 + 20:
            return (void*)&launch_step_pair<D2Q9, float, COLL_BGK, 32, 4>;
        case (ST_F32 * 2 + COLL_REG) * 32 + 10:
            return (void*)&launch_step_tma1<D2Q9, float, COLL_REG, 32, 4>;
        case (ST_F32 * 2 + COLL_REG) * 32 + 20:
            return (void*)&launch_step_pair<D2Q9, float, COLL_REG, 32, 4>;
        case (ST_BF16 * 2 + COLL_BGK) * 32 + 10:
            return (void*)&launch_step_tma1<D2Q9, __nv_bfloat16, COLL_BGK, 32, 4>;
        case (ST_BF16 * 2 + COLL_BGK) * 32 + 20:
            return (void*)&launch_step_pair<D2Q9, __nv_bfloat16, COLL_BGK, 32, 4>;
        case (ST_BF16 * 2 + COLL_REG) * 32 + 10:
            return (void*)&launch_step_tma1<D2Q9, __nv_bfloat16, COLL_REG, 32, 4>;
        case (ST_BF16 * 2 + COLL_REG) * 32 + 20:
            return (void*)&launch_step_pair<D2Q9, __nv_bfloat16, COLL_REG, 32, 4>;
        case (ST_F16 * 2 + COLL_BGK) * 32 + 10:
            return (void*)&launch_step_tma1<D2Q9, __half, COLL_BGK, 32, 4>;
        case (ST_F16 * 2 + COLL_BGK) * 32 + 20:
            return (void*)&launch_step_pair<D2Q9, __half, COLL_BGK, 32, 4>;
        case (ST_F16 * 2 + COLL_REG) * 32 + 10:
            return (void*)&launch_step_tma1<D2Q9, __half, COLL_REG, 32, 4>;
        case (ST_F16 * 2 + COLL_REG) * 32 + 20:
            return (void*)&launch_step_pair<D2Q9, __half, COLL_REG, 32, 4>;
        case (ST_F32 * 2 + COLL_BGK) * 32 + 27:
            return (void*)&launch_step_tman<D2Q9, float, COLL_BGK, 64, 1, 3, 12>;
        case (ST_F32 * 2 + COLL_REG) * 32 + 27:
            return (void*)&launch_step_tman<D2Q9, float, COLL_REG, 64, 1, 3, 12>;
        case (ST_BF16 * 2 + COLL_BGK) * 32 + 27:
            return (void*)&launch_step_tman<D2Q9, __nv_bfloat16, COLL_BGK, 64, 1, 3, 16>;
        case (ST_BF16 * 2 + COLL_REG) * 32 + 27:
            return (void*)&launch_step_tman<D2Q9, __nv_bfloat16, COLL_REG, 64, 1, 3, 16>;
        case (ST_F16 * 2 + COLL_BGK) * 32 + 27:
            return (void*)&launch_step_tman<D2Q9, __half, COLL_BGK, 64, 1, 3, 16>;
        case (ST_F16 * 2 + COLL_REG) * 32 + 27:
            return (void*)&launch_step_tman<D2Q9, __half, COLL_REG, 64, 1, 3, 16>;
        default:
            return nullptr;
    }
}

// Box of the staged kernels for a storage type and tile width bx: width (elements) and left pad.
void tma_box_q9(int storage, int bx, int* bw, int* pad) {
    switch (storage) {
        case ST_F32:
            *pad = TmaGeom<D2Q9, float, 2>::PAD;
            *bw = bx + 2 * *pad;
            return;
        case ST_BF16:
            *pad = TmaGeom<D2Q9, __nv_bfloat16, 2>::PAD;
            *bw = bx + 2 * *pad;
            return;
        case ST_F16:
            *pad = TmaGeom<D2Q9, __half, 2>::PAD;
            *bw = bx + 2 * *pad;
            return;
        default:
            *bw = *pad = 0;
    }
}

}  // namespace lbm
