// step_tma.cuh -- the fused step with TMA-staged, double-buffered tile loads (sm_103a).
//
// A persistent CTA walks tiles of BX x BY nodes.  For a tile that lies at least the lattice reach
// inside the grid, one thread issues Q bulk tensor copies (cp.async.bulk.tensor.3d, one box per
// direction plane): box i is the BY rows y0 - c_iy .. and the BX + 2 PAD columns x0 - PAD .., so
// it holds every pulled population h_i(x - c_i) of the tile.  The copies complete on an mbarrier;
// while they fly the CTA computes the previous tile (STAGES-deep ring).  Threads then read their
// populations from shared memory at compile-time offsets (no address arithmetic per direction),
// and run the same bounce-back, collision, store and force code as the plain kernel.  Tiles that
// touch the periodic edges use the plain wrapped global loads.  The arithmetic is the plain
// kernel's (same source), so results agree with it to FP32 rounding.
//
// Every wait on an mbarrier is bounded; a wait that runs out sets bit 2 of the error word, the
// CTA waits (again bounded) for its own copies in flight and returns.
#pragma once

#include <cuda.h>

#include "step_kernel.cuh"

namespace lbm {

template <class L, class ST, int STAGES_, int BX_ = 64, int BY_ = 4>
struct TmaGeom {
    static constexpr int BX = BX_, BY = BY_;
    static constexpr int THREADS = BX * BY;
    static constexpr int ES = (int)sizeof(ST);
    static constexpr int PAD = (16 / ES) >= L::R ? (16 / ES) : 2 * (16 / ES);  // 16-byte aligned, >= reach
    static constexpr int BW = BX + 2 * PAD;                                       // box width (elements)
    static constexpr int BOX_BYTES = BW * BY * ES;
    static constexpr int SLOT = (BOX_BYTES + 127) / 128 * 128;                    // one direction's box
    static constexpr int STAGE = L::Q * SLOT;
    static constexpr int STAGES = STAGES_;
    static constexpr int SMEM = STAGES * STAGE;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// Bulk tensor store of one box from shared memory (tracked by the thread's bulk async-group).
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int c0, int c1, int c2, const void* src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
                 : "memory");
}

constexpr long long kTmaWaitLimit = 4000000000ll;  // clock cycles (about 2 s)

// Tile t lies at least the lattice reach inside the grid (its boxes need no periodic wrap).
template <class G, class L>
__device__ __forceinline__ bool tile_interior(const InstDev& P, int t) {
    const int x0 = (t % P.ntx) * G::BX, y0 = (t / P.ntx) * G::BY;
    return x0 >= L::R && x0 + G::BX + L::R <= P.nx && y0 >= L::R && y0 + G::BY + L::R <= P.ny;
}

// Thread 0: arm the stage's barrier and issue the Q boxes of tile t.
template <class G, class L>
__device__ __forceinline__ void issue_tile(const InstDev& P, const CUtensorMap* map, int t, unsigned char* stage,
                                           uint64_t* bar) {
    const int x0 = (t % P.ntx) * G::BX, y0 = (t / P.ntx) * G::BY;
    mbar_expect_tx(bar, (unsigned)(L::Q * G::BOX_BYTES));
#pragma unroll
    for (int i = 0; i < L::Q; ++i) tma_load_3d(stage + i * G::SLOT, map, x0 - G::PAD, y0 - cy_of<L>(i), i, bar);
}

// Eq. 17 from a staged tile: h_i^adv = box_i[ty][tx + PAD - c_ix].
template <class G, class L, class ST>
__device__ __forceinline__ void gather_smem(const unsigned char* stage, int tx, int ty,
                                            typename StoreT<ST>::CT (&h)[L::Q]) {
    const ST* base = reinterpret_cast<const ST*>(stage) + ty * G::BW + tx + G::PAD;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const ST* p = reinterpret_cast<const ST*>(reinterpret_cast<const unsigned char*>(base) + i * G::SLOT) -
                      cx_of<L>(i);
        h[i] = StoreT<ST>::ld(p);
    }
}

// The tiles of one step of one instance, for a persistent CTA: tiles blockIdx.x, +gridDim.x, ...
// Returns false if a wait timed out (the CTA must return).
template <class L, class ST, int COLL, class G>
__device__ __forceinline__ bool run_tiles_tma(const InstDev& P, const CUtensorMap* map, const void* src, void* dst,
                                              double dv, float dv_f, double2* force_out, unsigned char* smem,
                                              uint64_t* bars, uint32_t& phase) {
    const int tid = threadIdx.y * G::BX + threadIdx.x;
    const int first = blockIdx.x, stride = gridDim.x;
    unsigned pending = 0;  // stages with copies in flight (thread 0's view)
    // prologue: the first STAGES-1 tiles of this CTA
    if (tid == 0) {
#pragma unroll
        for (int j = 0; j < G::STAGES - 1; ++j) {
            const int t = first + j * stride;
            if (t < P.ntiles && tile_interior<G, L>(P, t)) {
                issue_tile<G, L>(P, map, t, smem + j * G::STAGE, &bars[j]);
                pending |= 1u << j;
            }
        }
    }
    bool ok_all = true;
    int k = 0;
    for (int t = first; t < P.ntiles; t += stride, ++k) {
        const int s = k % G::STAGES;
        // refill the stage freed by the previous iteration with the tile STAGES-1 ahead
        if (tid == 0) {
            const int ks = (k + G::STAGES - 1) % G::STAGES;
            const int tn = t + (G::STAGES - 1) * stride;
            if (tn < P.ntiles && tile_interior<G, L>(P, tn)) {
                issue_tile<G, L>(P, map, tn, smem + ks * G::STAGE, &bars[ks]);
                pending |= 1u << ks;
            }
        }
        const int tx = t % P.ntx, ty = t / P.ntx;
        const int x = tx * G::BX + threadIdx.x;
        const int y = ty * G::BY + threadIdx.y;
        const int cls = (x < P.nx && y < P.ny) ? (int)P.cls[y * P.pitch + x] : (int)NODE_SOLID;
        double Fx = 0.0, Fy = 0.0;
        typename StoreT<ST>::CT h[L::Q];
        if (tile_interior<G, L>(P, t)) {
            const bool ok = mbar_wait(&bars[s], (phase >> s) & 1u, kTmaWaitLimit);
            phase ^= 1u << s;
            if (tid == 0) pending &= ~(1u << s);
            if (!__syncthreads_and(ok)) {
                ok_all = false;
                break;
            }
            if (cls != NODE_SOLID) {
                gather_smem<G, L, ST>(smem + s * G::STAGE, threadIdx.x, threadIdx.y, h);
                collide_store<L, ST, COLL>(P, src, dst, x, y, cls, dv, dv_f, h, Fx, Fy);
            }
        } else if (cls != NODE_SOLID) {
            gather_global<L, ST>(P, static_cast<const ST*>(src), x, y, h);
            collide_store<L, ST, COLL>(P, src, dst, x, y, cls, dv, dv_f, h, Fx, Fy);
        }
        tile_epilogue(P, P.tile_slot[t], force_out, Fx, Fy);
        __syncthreads();  // stage s may be refilled now
    }
    if (!ok_all) {
        if (tid == 0) {
            atomicOr(P.err, 4);
            // wait (bounded) for this CTA's own copies still in flight before its shared memory goes away
            for (int j = 0; j < G::STAGES; ++j)
                if (pending & (1u << j)) mbar_wait(&bars[j], (phase >> j) & 1u, kTmaWaitLimit);
        }
        __syncthreads();
        return false;
    }
    return true;
}

template <class G>
__device__ __forceinline__ void init_bars(uint64_t* bars) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
        for (int j = 0; j < G::STAGES; ++j) mbar_init(&bars[j], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
}

// Single-instance step, persistent CTAs over the tiles.
template <class L, class ST, int COLL, int STAGES>
__global__ void __launch_bounds__(256) step_kernel_tma(const __grid_constant__ InstDev P,
                                                       const __grid_constant__ CUtensorMap map) {
    using G = TmaGeom<L, ST, STAGES>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[STAGES];
    init_bars<G>(bars);
    uint32_t phase = 0;
    run_tiles_tma<L, ST, COLL, G>(P, &map, P.src, P.dst, P.dv, P.dv_f, P.force_out, smem, bars, phase);
}

// Single-instance step, one block per tile: an interior tile is staged by one set of Q bulk
// copies, waited for and computed; latency is hidden by the other resident blocks.
template <class L, class ST, int COLL, int BX, int BY>
__global__ void __launch_bounds__(BX * BY) step_kernel_tma1(const __grid_constant__ InstDev P,
                                                            const __grid_constant__ CUtensorMap map) {
    using G = TmaGeom<L, ST, 1, BX, BY>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    pdl_wait_then_release();  // before the tile's copies: they read the previous step's output
    const int t = blockIdx.x;
    const int slot = P.tile_slot[t];  // read early: the epilogue would otherwise wait for it
    const int tid = threadIdx.y * BX + threadIdx.x;
    const int x = (t % P.ntx) * BX + threadIdx.x;
    const int y = (t / P.ntx) * BY + threadIdx.y;
    const int cls = (x < P.nx && y < P.ny) ? (int)P.cls[y * P.pitch + x] : (int)NODE_SOLID;
    double Fx = 0.0, Fy = 0.0;
    typename StoreT<ST>::CT h[L::Q];
    if (tile_interior<G, L>(P, t)) {
        if (tid == 0) {
            mbar_init(&bar, 1);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_tile<G, L>(P, &map, t, smem, &bar);
        }
        __syncthreads();
        const bool ok = mbar_wait(&bar, 0, kTmaWaitLimit);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicOr(P.err, 4);
                mbar_wait(&bar, 0, kTmaWaitLimit);
            }
            __syncthreads();
            return;
        }
        if (cls != NODE_SOLID) {
            gather_smem<G, L, ST>(smem, threadIdx.x, threadIdx.y, h);
            collide_store<L, ST, COLL>(P, P.src, P.dst, x, y, cls, P.dv, P.dv_f, h, Fx, Fy);
        }
    } else if (cls != NODE_SOLID) {
        gather_global<L, ST>(P, static_cast<const ST*>(P.src), x, y, h);
        collide_store<L, ST, COLL>(P, P.src, P.dst, x, y, cls, P.dv, P.dv_f, h, Fx, Fy);
    }
    tile_epilogue(P, slot, P.force_out, Fx, Fy);
}

// Single-instance step, one block per tile of BX x (NR BY) nodes: the tile is staged by one set of
// Q bulk copies, and each thread computes NR nodes of its column, one row of BY apart at a time.
// The block's fixed costs (tile indices, launch constants, the copies and their barrier, the
// force epilogue) are spread over NR nodes per thread, while only one node's populations are live.
// MINB: resident blocks per SM the register allocation must allow (the compiler would otherwise keep
// launch constants live across the rows at the price of occupancy).
template <class L, class ST, int COLL, int BX, int BY, int NR, int MINB>
__global__ void __launch_bounds__(BX * BY, MINB) step_kernel_tman(const __grid_constant__ InstDev P,
                                                            const __grid_constant__ CUtensorMap map) {
    using G = TmaGeom<L, ST, 1, BX, BY * NR>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    // The geometry (tile slots, node classes) is written by the host only: it is read before the
    // wait for the previous step's grid, while that grid drains.
    const int t = blockIdx.x;
    const int slot = P.tile_slot[t];  // read early: the epilogue would otherwise wait for it
    const int tid = threadIdx.y * BX + threadIdx.x;
    const int x = (t % P.ntx) * BX + threadIdx.x;
    const int yt = (t / P.ntx) * (BY * NR);
    const bool interior = tile_interior<G, L>(P, t);
    int cls[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int y = yt + threadIdx.y + r * BY;
        cls[r] = (x < P.nx && y < P.ny) ? (int)P.cls[y * P.pitch + x] : (int)NODE_SOLID;
    }
    if (interior && tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    pdl_wait_then_release();  // before the tile's copies: they read the previous step's output
    if (interior) {
        if (tid == 0) issue_tile<G, L>(P, &map, t, smem, &bar);
        __syncthreads();
        const bool ok = mbar_wait(&bar, 0, kTmaWaitLimit);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicOr(P.err, 4);
                mbar_wait(&bar, 0, kTmaWaitLimit);
            }
            __syncthreads();
            return;
        }
    }
    double Fx = 0.0, Fy = 0.0;
#pragma unroll 1
    for (int r = 0; r < NR; ++r) {
        const int ty = threadIdx.y + r * BY;
        const int y = yt + ty;
        const int c = cls[0];
#pragma unroll
        for (int j = 0; j + 1 < NR; ++j) cls[j] = cls[j + 1];  // rotate: stays in registers
        if (c == NODE_SOLID) continue;
        typename StoreT<ST>::CT h[L::Q];
        if (interior)
            gather_smem<G, L, ST>(smem, threadIdx.x, ty, h);
        else
            gather_global<L, ST>(P, static_cast<const ST*>(P.src), x, y, h);
        collide_store<L, ST, COLL>(P, P.src, P.dst, x, y, c, P.dv, P.dv_f, h, Fx, Fy);
    }
    tile_epilogue(P, slot, P.force_out, Fx, Fy);
}

// Eq. 17 from a staged tile for the two neighbouring nodes (2 tx, 2 tx + 1) of a thread; a
// direction with even c_ix has both values in one aligned two-element word.
template <class G, class L, class ST>
__device__ __forceinline__ void gather_smem_pair(const unsigned char* stage, int tx, int ty,
                                                 typename StoreT<ST>::CT (&h0)[L::Q],
                                                 typename StoreT<ST>::CT (&h1)[L::Q]) {
    static_assert(G::PAD % 2 == 0 && G::BW % 2 == 0, "two-element words must stay aligned");
    const ST* base = reinterpret_cast<const ST*>(stage) + ty * G::BW + 2 * tx + G::PAD;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int cx = cx_of<L>(i);
        const ST* p = reinterpret_cast<const ST*>(reinterpret_cast<const unsigned char*>(base) + i * G::SLOT) - cx;
        if ((cx & 1) == 0) {
            StoreT<ST>::ld2(p, h0[i], h1[i]);
        } else {
            h0[i] = StoreT<ST>::ld(p);
            h1[i] = StoreT<ST>::ld(p + 1);
        }
    }
}

// Single-instance step, one block of TX x TY threads per tile of 2 TX x TY nodes; each thread
// updates the two neighbouring nodes (x, x + 1), x even, and stores both with one access per
// direction.  Interior tiles are staged by TMA; edge tiles read with wrapped global loads.
template <class L, class ST, int COLL, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) step_kernel_pair(const __grid_constant__ InstDev P,
                                                            const __grid_constant__ CUtensorMap map) {
    using G = TmaGeom<L, ST, 1, 2 * TX, TY>;
    using S = StoreT<ST>;
    using T = typename S::CT;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    pdl_wait_then_release();  // before the tile's copies: they read the previous step's output
    const int t = blockIdx.x;
    const int slot = P.tile_slot[t];  // read early: the epilogue would otherwise wait for it
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int x = (t % P.ntx) * (2 * TX) + 2 * threadIdx.x;
    const int y = (t / P.ntx) * TY + threadIdx.y;
    const bool row = y < P.ny;
    const int cls0 = (row && x < P.nx) ? (int)P.cls[y * P.pitch + x] : (int)NODE_SOLID;
    const int cls1 = (row && x + 1 < P.nx) ? (int)P.cls[y * P.pitch + x + 1] : (int)NODE_SOLID;
    double Fx = 0.0, Fy = 0.0;
    T h0[L::Q], h1[L::Q];
    if (tile_interior<G, L>(P, t)) {
        if (tid == 0) {
            mbar_init(&bar, 1);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_tile<G, L>(P, &map, t, smem, &bar);
        }
        __syncthreads();
        const bool ok = mbar_wait(&bar, 0, kTmaWaitLimit);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicOr(P.err, 4);
                mbar_wait(&bar, 0, kTmaWaitLimit);
            }
            __syncthreads();
            return;
        }
        gather_smem_pair<G, L, ST>(smem, threadIdx.x, threadIdx.y, h0, h1);
    } else {
        if (cls0 != NODE_SOLID) gather_global<L, ST>(P, static_cast<const ST*>(P.src), x, y, h0);
        if (cls1 != NODE_SOLID) gather_global<L, ST>(P, static_cast<const ST*>(P.src), x + 1, y, h1);
    }
    if (cls0 != NODE_SOLID || cls1 != NODE_SOLID) {
        Coef<T> C0, C1;
        if (cls0 != NODE_SOLID) prepare<L, ST, COLL>(P, P.src, x, y, cls0, P.dv, P.dv_f, h0, Fx, Fy, C0);
        if (cls1 != NODE_SOLID) prepare<L, ST, COLL>(P, P.src, x + 1, y, cls1, P.dv, P.dv_f, h1, Fx, Fy, C1);
        const bool f0 = cls0 != NODE_SOLID, f1 = cls1 != NODE_SOLID;
        ST* __restrict__ dst = static_cast<ST*>(P.dst) + y * P.pitch + x;
        const long long plane = P.plane;
        // solid nodes keep g = 0 (a stored 0 means h = H there; solid values are never read)
        S::st2(dst, f0 ? eval_rest<L, COLL, T>(C0, h0[0]) : (T)0, f1 ? eval_rest<L, COLL, T>(C1, h1[0]) : (T)0);
#pragma unroll
        for (int k = 0; k < L::NP; ++k) {
            T p0 = 0, m0 = 0, p1 = 0, m1 = 0;
            if (f0) eval_pair<L, COLL, T>(C0, k, h0[1 + 2 * k], h0[2 + 2 * k], p0, m0);
            if (f1) eval_pair<L, COLL, T>(C1, k, h1[1 + 2 * k], h1[2 + 2 * k], p1, m1);
            S::st2(dst + (1 + 2 * k) * plane, p0, p1);
            S::st2(dst + (2 + 2 * k) * plane, m0, m1);
        }
    }
    tile_epilogue(P, slot, P.force_out, Fx, Fy);
}

template <class L, class ST, int COLL, int TX, int TY>
cudaError_t launch_step_pair(const InstDev& P, const CUtensorMap& map, const CUtensorMap&, cudaStream_t stream) {
    using G = TmaGeom<L, ST, 1, 2 * TX, TY>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel_pair<L, ST, COLL, TX, TY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    return launch_pdl(step_kernel_pair<L, ST, COLL, TX, TY>, dim3(P.ntiles), dim3(TX, TY), G::SMEM, stream, P, map);
}

// Launch of a staged step: `map` addresses the source buffer with the load boxes, `store_map` the
// destination buffer with the tile's own box (used by the kernels that store through TMA).
using TmaStepLaunchFn = cudaError_t (*)(const InstDev& P, const CUtensorMap& map, const CUtensorMap& store_map,
                                        cudaStream_t stream);

template <class L, class ST, int COLL, int BX, int BY>
cudaError_t launch_step_tma1(const InstDev& P, const CUtensorMap& map, const CUtensorMap&, cudaStream_t stream) {
    using G = TmaGeom<L, ST, 1, BX, BY>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel_tma1<L, ST, COLL, BX, BY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    return launch_pdl(step_kernel_tma1<L, ST, COLL, BX, BY>, dim3(P.ntiles), dim3(BX, BY), G::SMEM, stream, P, map);
}

template <class L, class ST, int COLL, int BX, int BY, int NR, int MINB>
cudaError_t launch_step_tman(const InstDev& P, const CUtensorMap& map, const CUtensorMap&, cudaStream_t stream) {
    using G = TmaGeom<L, ST, 1, BX, BY * NR>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel_tman<L, ST, COLL, BX, BY, NR, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    return launch_pdl(step_kernel_tman<L, ST, COLL, BX, BY, NR, MINB>, dim3(P.ntiles), dim3(BX, BY), G::SMEM, stream,
                      P, map);
}

// The staged step with staged stores: an interior tile's outputs are written to a second
// shared-memory tile at compile-time offsets, then one thread stores each direction plane with one
// bulk tensor copy (box BX x BY at the tile's origin, never negative, x a multiple of BX) and waits
// for the copies before the block exits.  Nodes of the tile that are solid are stored as zero (no
// step ever reads them).  Tiles at the periodic edges keep the plain loads and stores.
template <class L, class ST, int COLL, int BX, int BY>
struct TmaStoreGeom {
    using G = TmaGeom<L, ST, 1, BX, BY>;
    static constexpr int OSLOT = (BX * BY * (int)sizeof(ST) + 127) / 128 * 128;  // one plane of outputs
    static constexpr int SMEM = G::SMEM + L::Q * OSLOT;
};

template <class L, class ST, int COLL, int BX, int BY>
__global__ void __launch_bounds__(BX * BY) step_kernel_tma1s(const __grid_constant__ InstDev P,
                                                             const __grid_constant__ CUtensorMap map,
                                                             const __grid_constant__ CUtensorMap smap) {
    using G = TmaGeom<L, ST, 1, BX, BY>;
    using O = TmaStoreGeom<L, ST, COLL, BX, BY>;
    using S = StoreT<ST>;
    using T = typename S::CT;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    pdl_wait_then_release();  // before the tile's copies: they read the previous step's output
    const int t = blockIdx.x;
    const int slot = P.tile_slot[t];  // read early: the epilogue would otherwise wait for it
    const int tid = threadIdx.y * BX + threadIdx.x;
    const int x = (t % P.ntx) * BX + threadIdx.x;
    const int y = (t / P.ntx) * BY + threadIdx.y;
    const int cls = (x < P.nx && y < P.ny) ? (int)P.cls[y * P.pitch + x] : (int)NODE_SOLID;
    double Fx = 0.0, Fy = 0.0;
    T h[L::Q];
    if (tile_interior<G, L>(P, t)) {
        if (tid == 0) {
            mbar_init(&bar, 1);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_tile<G, L>(P, &map, t, smem, &bar);
        }
        __syncthreads();
        const bool ok = mbar_wait(&bar, 0, kTmaWaitLimit);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicOr(P.err, 4);
                mbar_wait(&bar, 0, kTmaWaitLimit);
            }
            __syncthreads();
            return;
        }
        unsigned char* out = smem + G::SMEM;
        const int o = threadIdx.y * BX + threadIdx.x;
        if (cls != NODE_SOLID) {
            gather_smem<G, L, ST>(smem, threadIdx.x, threadIdx.y, h);
            collide_emit<L, ST, COLL>(P, P.src, x, y, cls, P.dv, P.dv_f, h, Fx, Fy,
                                      [&](int i, T v) { S::st(reinterpret_cast<ST*>(out + i * O::OSLOT) + o, v); });
        } else {
#pragma unroll
            for (int i = 0; i < L::Q; ++i) S::st(reinterpret_cast<ST*>(out + i * O::OSLOT) + o, (T)0);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> async proxy
        __syncthreads();
        if (tid == 0) {
            const int x0 = (t % P.ntx) * BX, y0 = (t / P.ntx) * BY;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) tma_store_3d(&smap, x0, y0, i, out + i * O::OSLOT);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            // the block may exit once the copies have read its shared memory; the global writes
            // complete with the grid
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        }
    } else if (cls != NODE_SOLID) {
        gather_global<L, ST>(P, static_cast<const ST*>(P.src), x, y, h);
        collide_store<L, ST, COLL>(P, P.src, P.dst, x, y, cls, P.dv, P.dv_f, h, Fx, Fy);
    }
    tile_epilogue(P, slot, P.force_out, Fx, Fy);
}

template <class L, class ST, int COLL, int BX, int BY>
cudaError_t launch_step_tma1s(const InstDev& P, const CUtensorMap& map, const CUtensorMap& smap,
                              cudaStream_t stream) {
    using O = TmaStoreGeom<L, ST, COLL, BX, BY>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel_tma1s<L, ST, COLL, BX, BY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, O::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    return launch_pdl(step_kernel_tma1s<L, ST, COLL, BX, BY>, dim3(P.ntiles), dim3(BX, BY), O::SMEM, stream, P, map,
                      smap);
}

// Launch with one CTA per SM slot the kernel's shared memory allows (at most one per tile).
template <class L, class ST, int COLL, int STAGES>
cudaError_t launch_step_tma(const InstDev& P, const CUtensorMap& map, const CUtensorMap&, cudaStream_t stream) {
    using G = TmaGeom<L, ST, STAGES>;
    static int grid_cap = 0;  // per instantiation: SMs x resident CTAs
    if (!grid_cap) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel_tma<L, ST, COLL, STAGES>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0, dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel_tma<L, ST, COLL, STAGES>,
                                                                 G::THREADS, G::SMEM)) != cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid_cap = per_sm * sms;
    }
    const int grid = P.ntiles < grid_cap ? P.ntiles : grid_cap;
    step_kernel_tma<L, ST, COLL, STAGES><<<grid, dim3(G::BX, G::BY), G::SMEM, stream>>>(P, map);
    return cudaGetLastError();
}

}  // namespace lbm
