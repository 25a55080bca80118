// pbatch.cuh -- the persistent batched step: one launch advances many lattice instances of uneven
// sizes by K time steps, with no grid-wide barrier.
//
// Work items are (batch step k, strip) pairs in step-major order.  A strip is one tile column of a
// band of S tile rows of one instance; the strips of a band follow each other in the list.  Blocks
// take items from a global counter (one atomic per item, taken when the block is ready to start
// it), so the strips of a band start together and walk down their columns side by side:
// horizontally neighbouring tiles, whose staged boxes overlap by the lattice reach (and by the
// 32-byte sectors around it), are read at about the same time and share those reads in L2.  (An
// item index fetched one item ahead decorrelates the start of neighbouring strips by up to one
// item's duration, long enough for the shared sectors to leave L2: 1.4x the algorithmic DRAM reads
// against 1.1x.)  A strip of local step n + 1 waits only for the bands of its own instance within
// the lattice reach of its band to have finished step n: that one condition covers both the
// populations it reads (written at step n) and the ones it overwrites (read at step n by those
// neighbours).  Each band counts its finished strips in a per-instance array (band b has finished
// step n when its count reaches (n + 1) x tile columns).  Because items are taken in step-major
// order, every item a strip waits for was taken earlier by a running block, so the wait always
// ends; no co-residency of the grid is needed.
//
// The force of a step is reduced as in the single-instance kernels (per-tile FP64 slot, fixed-
// order sum by the last slot tile), into a ring of force slots indexed by n mod kRing, so that
// tiles of different steps of one instance can be in flight at once; an item of an instance with
// body links first waits for the sum of step n - kRing to have left its ring entry.
//
// Every wait is bounded: a wait that runs out sets a bit of the error word and the block returns
// (the blocks waiting on its items then run out too); the host reports LBM_ETIMEOUT.
//
// The tile code is that of the single-instance kernels (staged TMA tiles of BX x NR nodes, one
// thread per column, or plain tiles of 32 x 4 nodes with global loads), so every instance is
// computed exactly as lbm_step computes it with the same tile shape.  The populations other blocks
// of the launch wrote are read after an acquire of their band counters: by TMA (after a proxy
// fence) or by plain weak loads, never through the read-only path.
#pragma once

#include <cuda.h>
#include <stddef.h>

#include "step_tma.cuh"

namespace lbm {

constexpr int kRing = 4;  // steps of one instance whose forces may be in flight together

// Per-step constants of one instance, tabulated by the host: the drive of the step and the
// 16-bit stream-offset constants (see InstDev).
struct StepConst {
    double dv;
    float dv_f;
    float H[28];  // HM[6], Hl[7], Hs[7], He[4], Ho[4], in InstDev's order
    float pad;
};
static_assert(sizeof(StepConst) == 128, "one step's constants are one 128-byte line");
static_assert(offsetof(InstDev, Ho) + 4 * sizeof(float) - offsetof(InstDev, HM) == 28 * sizeof(float),
              "the stream-offset constants of InstDev are 28 contiguous floats");
static_assert(sizeof(InstDev) % 8 == 0, "InstDev is copied as 8-byte words");

// One instance of a persistent launch.
struct alignas(64) PInst {
    CUtensorMap maps[2];       // staged loads of buf[0] and buf[1] (boxes of the tile shape)
    InstDev base;              // geometry and constants (src, dst, dv, force scratch set per item)
    const void* buf[2];        // population buffers; local step n reads buf[n & 1]
    const StepConst* steps;    // [nsteps]
    double2* history;          // [nsteps] force of each local step
    int* done;                 // [bands] strips of each band completed, over all steps
    double2* ring;             // [kRing][nslots] force partials
    unsigned int* tickets;     // [kRing] slot tiles of the ring entry's step that have finished
    int* fin;                  // [kRing] 1 + the last step whose force left the entry
    long long start;           // batch step at which local step 0 runs
    long long nsteps;          // local steps to run
    int nty;                   // tiles along y
    int bx, by;                // tile shape in nodes
    int band;                  // tile rows per band (the tiles of one strip)
    int nseg;                  // strips per band (tile columns)
};

enum PbPath { PB_STAGED = 0, PB_PLAIN = 1 };

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bands of an instance (bands of h >= R nodes along a periodic axis of ny nodes, the last one
// possibly shorter) that hold a node within reach R of band b, each listed once: at most four (R
// nodes on either side span at most two bands, the short last one and its neighbour).
__device__ __forceinline__ int halo_bands(int band, int h, int ny, int R, int (&out)[4]) {
    const int first = band * h - R;                   // first node of the halo (>= -R)
    const int last = min(band * h + h, ny) - 1 + R;   // last node (< ny + h + R)
    int k = 0;
    for (int c = first; c <= last && k < 4;) {
        int cw = c % ny;
        if (cw < 0) cw += ny;
        const int bb = cw / h;
        bool seen = false;
        for (int j = 0; j < k; ++j) seen = seen || out[j] == bb;
        if (!seen) out[k++] = bb;
        c += min((bb + 1) * h, ny) - cw;  // first node of the next band
    }
    return k;
}

// Warp 0: wait until every band within reach of band b of the instance has completed local step
// n - 1, i.e. counted n x nseg strips (lanes 0-3, one band each; only for n >= 1), and until the
// sum of the force of step n - kRing has left ring entry n mod kRing (lane 4; instances with body
// links, n >= kRing).
// Returns false (in every lane) if a wait ran out.
template <class L>
__device__ __forceinline__ bool wait_item(const PInst& I, int band, long long n, long long limit) {
    int bands[4];
    const int nb = n > 0 ? halo_bands(band, I.band * I.by, I.base.ny, L::R, bands) : 0;
    const int lane = threadIdx.x & 31;
    const int* p = nullptr;
    int need = 0;
    if (lane < nb) {
        int b = bands[0];
#pragma unroll
        for (int j = 1; j < 4; ++j)
            if (lane == j) b = bands[j];
        p = I.done + b;
        need = (int)n * I.nseg;
    } else if (lane == 4 && I.base.nslots > 0 && n >= kRing) {
        p = I.fin + (int)(n % kRing);
        need = (int)(n - kRing + 1);
    }
    bool ok = true;
    if (p) {
        const long long t0 = clock64();
        while (true) {
            if (clock64() - t0 >= limit) {  // the clock first: a limit of 0 gives up at once
                ok = false;
                break;
            }
            if (ld_acquire(p) >= need) break;
            __nanosleep(32);
        }
    }
    return __all_sync(0xffffffffu, ok);
}

// Launch parameters of the persistent kernel.
struct PbArgs {
    const PInst* insts;
    const int4* segs;             // (instance, band, tile column, 0) of every strip
    int nsegs;                    // strips per batch step
    int nsteps;                   // batch steps of this launch
    long long step0;              // batch step of the launch's first step
    unsigned long long* queue;    // item counter (monotonic over launches)
    unsigned long long base;      // its value when this launch started
    int* err;                     // bit 3: a wait ran out
    long long limit;              // clock cycles a wait may take
};

template <class L, class ST, int COLL, int PATH, int BX, int NR, int MINB>
struct PbShape {
    static constexpr int THREADS = PATH == PB_STAGED ? BX : 128;
    static constexpr int TX = PATH == PB_STAGED ? BX : 32;   // tile in nodes
    static constexpr int TY = PATH == PB_STAGED ? NR : 4;
    using G = TmaGeom<L, ST, 1, BX, NR>;
    static constexpr int SMEM = PATH == PB_STAGED ? G::SMEM : 0;
};

template <class L, class ST, int COLL, int PATH, int BX, int NR, int MINB>
__global__ void __launch_bounds__(PbShape<L, ST, COLL, PATH, BX, NR, MINB>::THREADS, MINB)
    pbatch_kernel(const __grid_constant__ PbArgs A) {
    using Sh = PbShape<L, ST, COLL, PATH, BX, NR, MINB>;
    using G = typename Sh::G;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(16) InstDev P;   // the item's instance, with this step's constants
    __shared__ unsigned long long s_next;
    __shared__ int s_fail;
    // what the tiles of the current item need besides P (kept here, not in registers)
    __shared__ const CUtensorMap* s_map;
    __shared__ double2* s_force;   // force of this step in the instance's history
    __shared__ int* s_fin;         // ring entry's finish mark
    __shared__ int s_fin_val;      // value it takes when this step's force is written
    __shared__ int s_inst;         // instance and local step whose constants P holds
    __shared__ long long s_n;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;
    const unsigned long long total = (unsigned long long)A.nsteps * (unsigned long long)A.nsegs;
    if (tid == 0) {
        if (PATH == PB_STAGED) {
            mbar_init(&bar, 1);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        s_fail = 0;
        s_inst = -1;
        s_n = -1;
    }
    uint32_t parity = 0;
    while (true) {
        __syncthreads();  // the previous item is finished and every thread has read s_next
        if (tid == 0) s_next = atomicAdd(A.queue, 1ull) - A.base;
        __syncthreads();
        const unsigned long long w = s_next;
        if (w >= total) break;
        const int k = (int)(w / (unsigned)A.nsegs);
        const int4 it = A.segs[w - (unsigned long long)k * (unsigned)A.nsegs];
        const PInst& I = A.insts[it.x];
        const long long n = A.step0 + k - I.start;
        if (n < 0 || n >= I.nsteps) continue;  // block-uniform: the instance does not run this step
        const int band = it.y, tx = it.z;
        const int ring = (int)(n % kRing);
        const bool fresh = it.x != s_inst || n != s_n;  // P holds another instance or step
        // dependencies (warp 0, wait_item); the other warps meanwhile copy the instance's constants
        // into shared memory
        if (tid < 32) {
            const bool ok = wait_item<L>(I, band, n, A.limit);
            if (!ok && tid == 0) {
                atomicOr(A.err, 8);
                s_fail = 1;
            }
        }
        if (fresh) {
            const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&I.base);
            unsigned long long* dst = reinterpret_cast<unsigned long long*>(&P);
            constexpr int W = (int)(sizeof(InstDev) / 8);
            for (int j = tid; j < W; j += nthreads) dst[j] = src[j];
        }
        __syncthreads();
        if (s_fail) break;
        if (!fresh) {
            // same instance and step as the previous item: only the staged boxes need the fence
        } else if (tid < 28) {
            reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(&P) + offsetof(InstDev, HM))[tid] =
                I.steps[n].H[tid];
        } else if (tid == nthreads - 1) {
            const StepConst& S = I.steps[n];
            P.dv = S.dv;
            P.dv_f = S.dv_f;
            P.src = I.buf[n & 1];
            P.dst = const_cast<void*>(I.buf[(n + 1) & 1]);
            P.partials = I.ring + (size_t)ring * (size_t)(I.base.nslots > 0 ? I.base.nslots : 1);
            P.ticket = I.tickets + ring;
            s_map = &I.maps[n & 1];
            s_force = I.history + n;
            s_fin = I.fin + ring;
            s_fin_val = (int)(n + 1);
            s_inst = it.x;
            s_n = n;
        }
        // the staged tiles' boxes read what other blocks wrote through the generic proxy, made
        // visible to this block by warp 0's acquire: order the async proxy after it, once per item
        if (PATH == PB_STAGED && tid == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
        __syncthreads();
        const int ntx = P.ntx;
        const int ty0 = band * I.band, ty1 = min(ty0 + I.band, I.nty);
        for (int ty = ty0; ty < ty1; ++ty) {
            const int t = ty * ntx + tx;
            const int slot = P.tile_slot[t];
            double Fx = 0.0, Fy = 0.0;
            if constexpr (PATH == PB_STAGED) {
                const int x = tx * BX + threadIdx.x;
                const int yt = ty * NR;
                int cls[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int y = yt + r;
                    cls[r] = (x < P.nx && y < P.ny) ? (int)P.cls[y * P.pitch + x] : (int)NODE_SOLID;
                }
                const bool interior = tile_interior<G, L>(P, t);
                if (interior) {
                    if (tid == 0) issue_tile<G, L>(P, s_map, t, smem, &bar);
                    const bool ok = mbar_wait(&bar, parity, kTmaWaitLimit);
                    parity ^= 1u;
                    if (!__syncthreads_and(ok)) {
                        if (tid == 0) {
                            atomicOr(P.err, 4);
                            mbar_wait(&bar, parity ^ 1u, kTmaWaitLimit);
                        }
                        __syncthreads();
                        return;
                    }
                }
#pragma unroll 1
                for (int r = 0; r < NR; ++r) {
                    const int y = yt + r;
                    const int c = cls[0];
#pragma unroll
                    for (int j = 0; j + 1 < NR; ++j) cls[j] = cls[j + 1];
                    if (c == NODE_SOLID) continue;
                    typename StoreT<ST>::CT h[L::Q];
                    if (interior)
                        gather_smem<G, L, ST>(smem, threadIdx.x, r, h);
                    else
                        gather_global<L, ST, true>(P, static_cast<const ST*>(P.src), x, y, h);
                    collide_store<L, ST, COLL, 0, true>(P, P.src, P.dst, x, y, c, P.dv, P.dv_f, h, Fx, Fy);
                }
            } else {
                const int x = tx * 32 + threadIdx.x;
                const int y = ty * 4 + threadIdx.y;
                if (x < P.nx && y < P.ny) {
                    const int c = (int)P.cls[y * P.pitch + x];
                    if (c != NODE_SOLID) {
                        typename StoreT<ST>::CT h[L::Q];
                        gather_global<L, ST, true>(P, static_cast<const ST*>(P.src), x, y, h);
                        collide_store<L, ST, COLL, 0, true>(P, P.src, P.dst, x, y, c, P.dv, P.dv_f, h, Fx, Fy);
                    }
                }
            }
            if (tile_epilogue(P, slot, s_force, Fx, Fy) && tid == 0) {
                __threadfence();
                st_release(s_fin, s_fin_val);
            }
            if (PATH == PB_STAGED) __syncthreads();  // the stage is free for the next tile
        }
        __syncthreads();  // every store of the strip issued
        if (tid == 0) {
            __threadfence();
            atomicAdd(A.insts[it.x].done + band, 1);
        }
    }
}

using PbLaunchFn = cudaError_t (*)(const PbArgs& a, int grid, cudaStream_t stream);

// Kernel function, block shape and shared memory of one persistent-kernel instantiation, so that
// the host can put its launch into a CUDA graph node.
struct PbKernel {
    const void* func;
    dim3 block;
    int smem;
    int tile_x, tile_y;
};

template <class L, class ST, int COLL, int PATH, int BX, int NR, int MINB>
PbKernel pbatch_kernel_info() {
    using Sh = PbShape<L, ST, COLL, PATH, BX, NR, MINB>;
    PbKernel k;
    k.func = (const void*)&pbatch_kernel<L, ST, COLL, PATH, BX, NR, MINB>;
    k.block = PATH == PB_STAGED ? dim3(BX, 1) : dim3(32, 4);
    k.smem = Sh::SMEM;
    k.tile_x = Sh::TX;
    k.tile_y = Sh::TY;
    return k;
}

// The persistent kernel of a (lattice, storage, collision) class, by the variant whose tile code it
// runs (lbm_set_variant numbers): 27 = staged 64 x 3 tiles, 28 = staged 128 x 3 tiles (D2Q37),
// 2 = plain 32 x 4 tiles (D2Q37, 4- and 2-byte storage), 0 = plain 32 x 4 tiles (the others);
// func is null if not built.
PbKernel find_pbatch_kernel(int Q, int storage, int coll, int variant);

}  // namespace lbm
