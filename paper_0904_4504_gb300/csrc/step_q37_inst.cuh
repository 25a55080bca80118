// D2Q37 launch tables for one storage type: each of step_q37_f64.cu, step_q37_f32.cu,
// step_q37_bf16.cu and step_q37_f16.cu instantiates them for its type (four translation units that
// compile in parallel).  Variant numbers are those of lbm_set_variant.
#pragma once

#include "pbatch.cuh"

namespace lbm {

// Plain step, bounce-back walls.
template <class ST>
void* q37_plain(int coll) {
    if (coll == COLL_REG) return (void*)&launch_step<D2Q37, ST, COLL_REG>;
    if (coll == COLL_BGK) return (void*)&launch_step<D2Q37, ST, COLL_BGK>;
    return nullptr;
}

// The persistent batch kernel (pbatch.cuh), by the variant whose tile code it runs: 27 = staged
// 64 x 3 tiles (16-bit storage: 11 blocks of 64 threads per SM; FP32: 6, as shared memory allows),
// 28 = staged 128 x 3 tiles (6 blocks of 128 threads), 2 = plain 32 x 4 tiles (6 blocks of 128
// threads per SM, the register budget of variant 1), 0 = plain 32 x 4 tiles for FP64 (3 blocks).
template <class ST, int COLL>
PbKernel q37_pbatch_c(int variant) {
    constexpr bool wide = sizeof(ST) == 8;
    if constexpr (!wide) {
        if (variant == 27)
            return pbatch_kernel_info<D2Q37, ST, COLL, PB_STAGED, 64, 3, sizeof(ST) == 2 ? 11 : 6>();
        if (variant == 28) return pbatch_kernel_info<D2Q37, ST, COLL, PB_STAGED, 128, 3, sizeof(ST) == 2 ? 6 : 3>();
        if (variant == 2) return pbatch_kernel_info<D2Q37, ST, COLL, PB_PLAIN, 32, 4, 6>();
    } else {
        if (variant == 0) return pbatch_kernel_info<D2Q37, ST, COLL, PB_PLAIN, 32, 4, 3>();
    }
    return PbKernel{nullptr, dim3(), 0, 0, 0};
}

template <class ST>
PbKernel q37_pbatch(int coll, int variant) {
    if (coll == COLL_REG) return q37_pbatch_c<ST, COLL_REG>(variant);
    if (coll == COLL_BGK) return q37_pbatch_c<ST, COLL_BGK>(variant);
    return PbKernel{nullptr, dim3(), 0, 0, 0};
}

// Plain step with diffuse-scattering walls.
template <class ST>
void* q37_plain_ds(int coll) {
    if (coll == COLL_REG) return (void*)&launch_step<D2Q37, ST, COLL_REG, 1>;
    if (coll == COLL_BGK) return (void*)&launch_step<D2Q37, ST, COLL_BGK, 1>;
    return nullptr;
}

// Plain step with an occupancy floor: variant 1 = 6, 2 = 7 blocks of 128 threads per SM; 3, 4 = 7
// blocks, each thread computing 2 or 4 nodes of its column (tiles of 32 x 8, 32 x 16 nodes).
template <class ST, int COLL>
void* q37_occ_c(int variant) {
    switch (variant) {
        case 1: return (void*)&launch_step_occ<D2Q37, ST, COLL, 6>;
        case 2: return (void*)&launch_step_occ<D2Q37, ST, COLL, 7>;
        case 3: return (void*)&launch_step_occn<D2Q37, ST, COLL, 7, 2>;
        case 4: return (void*)&launch_step_occn<D2Q37, ST, COLL, 7, 4>;
        default: return nullptr;
    }
}

// Staged steps (tiles in nodes): 10, 11, 12 = one node per thread on 32 x 4, 64 x 2, 64 x 4 tiles;
// 13 = 64 x 2 with the outputs stored through TMA; 18, 23, 24, 25 = several nodes per thread, one
// row apart: blocks of 64 x 1 (4 rows), 64 x 1 (2 rows), 64 x 1 (4 rows, 10 blocks per SM),
// 128 x 1 (2 rows) threads; 26, 27 = 64 x 1 threads, 3 rows, at least 12 or 11 blocks per SM;
// 28 = 128 x 1 threads, 3 rows, 6 blocks per SM.
template <class ST, int COLL>
void* q37_tma_c(int variant) {
    switch (variant) {
        case 10: return (void*)&launch_step_tma1<D2Q37, ST, COLL, 32, 4>;
        case 11: return (void*)&launch_step_tma1<D2Q37, ST, COLL, 64, 2>;
        case 12: return (void*)&launch_step_tma1<D2Q37, ST, COLL, 64, 4>;
        case 13: return (void*)&launch_step_tma1s<D2Q37, ST, COLL, 64, 2>;
        case 18: return (void*)&launch_step_tman<D2Q37, ST, COLL, 64, 1, 4, 12>;
        case 23: return (void*)&launch_step_tman<D2Q37, ST, COLL, 64, 1, 2, 12>;
        case 24: return (void*)&launch_step_tman<D2Q37, ST, COLL, 64, 1, 4, 10>;
        case 25: return (void*)&launch_step_tman<D2Q37, ST, COLL, 128, 1, 2, 6>;
        case 26: return (void*)&launch_step_tman<D2Q37, ST, COLL, 64, 1, 3, 12>;
        case 27: return (void*)&launch_step_tman<D2Q37, ST, COLL, 64, 1, 3, 11>;
        case 28: return (void*)&launch_step_tman<D2Q37, ST, COLL, 128, 1, 3, 6>;
        default: return nullptr;
    }
}

template <class ST>
void* q37_occ(int coll, int variant) {
    return coll == COLL_REG ? q37_occ_c<ST, COLL_REG>(variant) : coll == COLL_BGK ? q37_occ_c<ST, COLL_BGK>(variant)
                                                                                    : nullptr;
}

template <class ST>
void* q37_tma(int coll, int variant) {
    return coll == COLL_REG ? q37_tma_c<ST, COLL_REG>(variant) : coll == COLL_BGK ? q37_tma_c<ST, COLL_BGK>(variant)
                                                                                    : nullptr;
}

// Box of the staged kernels for tile width bx: width (elements) and left pad.
template <class ST>
void q37_box(int bx, int* bw, int* pad) {
    *pad = TmaGeom<D2Q37, ST, 1>::PAD;
    *bw = bx + 2 * *pad;
}

}  // namespace lbm

// The functions one translation unit exports for storage type ST under the suffix SFX.
#define LBM_Q37_EXPORTS(SFX, ST, STAGED)                                                                 \
    namespace lbm {                                                                                      \
    void* find_launcher_q37_##SFX(int coll) { return q37_plain<ST>(coll); }                           \
    PbKernel find_pbatch_q37_##SFX(int coll, int variant) { return q37_pbatch<ST>(coll, variant); }    \
    void* find_launcher_q37_##SFX##_ds(int coll) { return q37_plain_ds<ST>(coll); }                    \
    void* find_occ_launcher_q37_##SFX(int coll, int variant) {                                          \
        return STAGED ? q37_occ<ST>(coll, variant) : nullptr;                                            \
    }                                                                                                    \
    void* find_tma_launcher_q37_##SFX(int coll, int variant) {                                          \
        return STAGED ? q37_tma<ST>(coll, variant) : nullptr;                                            \
    }                                                                                                    \
    void tma_box_q37_##SFX(int bx, int* bw, int* pad) {                                                 \
        if (STAGED) q37_box<ST>(bx, bw, pad);                                                            \
        else *bw = *pad = 0;                                                                             \
    }                                                                                                    \
    }
