// In-place streaming on one population buffer (the "AA" access pattern).
//
// Two lattice steps of Eqs. 17-18 take two kernels that read and write the same buffer A:
//
//   step n (even):  pull h_i(x - c_i) from plane opp(i) (where the previous local step left the
//                   post-collision values, directions swapped), bounce back from the node's own
//                   plane i, collide, and push each output to A[x + c_i][i]; an output whose link
//                   x -> x + c_i is blocked comes straight back into A[x][opp(i)] with the wall
//                   term of step n + 1, so the next step needs no fix-up.
//   step n+1 (odd): read the node's own A[x][i] (already streamed), collide, and store output i
//                   into A[x][opp(i)].
//
// Every node of a step reads and writes the same set of slots, and no two nodes share a slot (a
// slot read across a link is never the one a blocked link reads at home), so the update is in
// place without races; every store of a node depends on all of its loads (through the moments),
// so no store can overtake a load of the same slot.  After an even number of steps A holds the post-collision state with
// directions swapped.  The bytes per lattice update are those of the two-buffer step (one read and
// one write per population); the population footprint is halved.
//
// The momentum exchange of a bounced link belongs to the step that pulls it.  The pull-push kernel
// therefore records two forces: that of step n (links bounced on the pull) and that of step n + 1
// (links bounced on the push, with the wall term of step n + 1); the local kernel records none.
#pragma once

#include "step_kernel.cuh"

namespace lbm {

// Rows and columns y - d, x - d (d = -R..R, periodic) around node (x, y): the pull source x - c_i
// of direction i is (roff[cy + R], col[cx + R]) and its push target x + c_i is (roff[R - cy],
// col[R - cx]), so one table serves both.
template <int R>
__device__ __forceinline__ void neighbour_table(const InstDev& P, int x, int y, int (&roff)[2 * R + 1],
                                                int (&col)[2 * R + 1]) {
#pragma unroll
    for (int d = -R; d <= R; ++d) {
        int ys = y - d;
        ys += ys < 0 ? P.ny : 0;
        ys -= ys >= P.ny ? P.ny : 0;
        int xs = x - d;
        xs += xs < 0 ? P.nx : 0;
        xs -= xs >= P.nx ? P.nx : 0;
        roff[d + R] = ys * P.pitch;
        col[d + R] = xs;
    }
}

// Collision outputs of one node pushed to their targets.  BND: the node has blocked links, and an
// output whose link x -> x + c_i is blocked (exactly when pull link opp(i) is) comes back into the
// node's own slot A[x][opp(i)] with the wall term of step n + 1; its momentum exchange goes to
// (Gx, Gy), the force of step n + 1.  Bulk nodes push every output without tests.
template <class L, class ST, int COLL, bool BND>
__device__ __forceinline__ void aa_push(const InstDev& P, ST* A, int idx, const int (&roff)[2 * L::R + 1],
                                        const int (&col)[2 * L::R + 1], const Coef<typename StoreT<ST>::CT>& C,
                                        const typename StoreT<ST>::CT (&h)[L::Q], double& Gx, double& Gy) {
    using S = StoreT<ST>;
    using T = typename S::CT;
    constexpr int R = L::R;
    const long long plane = P.plane;
    const bool off = sizeof(ST) == 2 && P.stream_off;
    ulonglong2 lk = make_ulonglong2(0ull, 0ull);
    if (BND) lk = P.links[idx];
    const unsigned long long blk = lk.x | lk.y;

    // v: output i relative to the stored state's stream offset (16-bit), as eval_pair returns it
    auto push = [&](int i, T v) {
        const int j = opp_of<L>(i);
        if (BND && ((blk >> j) & 1ull)) {
            double mw = 0.0;
            const T hi = off ? (T)off_s<L>(P, i) : (T)0;
            if ((lk.x >> j) & 1ull) {
                if (P.moving) mw = P.mw_k * cx_of<L>(j) * P.dv2;
                // the value the two-buffer step would read back: v rounded to the storage type
                const T own = S::rnd(v) + hi;
                const double hs = 2.0 * (double)own + mw;
                const double ws = w_of<L>(j) * P.s;
                Gx -= cx_of<L>(j) * ws * hs;
                Gy -= cy_of<L>(j) * ws * hs;
            }
            S::st(A + j * plane + idx, v + hi + (T)mw - (off ? (T)off_s<L>(P, j) : (T)0));
        } else {
            S::st(A + i * plane + roff[R - cy_of<L>(i)] + col[R - cx_of<L>(i)], v);
        }
    };
    emit_outputs<L, ST, COLL>(C, h, [&](int i, T v) {
        if (i == 0)
            S::st(A + idx, v);
        else
            push(i, v);
    });
}

// Even step of one node: pull h_i = A[x - c_i][opp(i)], wall fix-up from the node's own plane i,
// collide, push.  (Fx, Fy) gets the force of step n, (Gx, Gy) that of step n + 1.  The neighbour
// table is built twice, for the pull and again for the push, rather than kept live through the
// collision (registers).
template <class L, class ST, int COLL>
__device__ __forceinline__ void aa_pull_push(const InstDev& P, ST* A, int x, int y, int cls, double& Fx,
                                             double& Fy, double& Gx, double& Gy) {
    using S = StoreT<ST>;
    using T = typename S::CT;
    constexpr int Q = L::Q, R = L::R;
    const long long plane = P.plane;
    const int idx = y * P.pitch + x;
    T h[Q];
    {
        int roff[2 * R + 1], col[2 * R + 1];
        neighbour_table<R>(P, x, y, roff, col);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            h[i] = S::ld(A + opp_of<L>(i) * plane + roff[cy_of<L>(i) + R] + col[cx_of<L>(i) + R]);
    }
    Coef<T> C;
    prepare<L, ST, COLL, 0, OWN_SWAPPED>(P, A, x, y, cls, P.dv, P.dv_f, h, Fx, Fy, C);
    int roff[2 * R + 1], col[2 * R + 1];
    neighbour_table<R>(P, x, y, roff, col);
    if (cls == NODE_BOUNDARY)
        aa_push<L, ST, COLL, true>(P, A, idx, roff, col, C, h, Gx, Gy);
    else
        aa_push<L, ST, COLL, false>(P, A, idx, roff, col, C, h, Gx, Gy);
}

// Odd step of one node: local read, collide, store directions swapped.
template <class L, class ST, int COLL>
__device__ __forceinline__ void aa_local(const InstDev& P, ST* A, int x, int y, int cls) {
    using S = StoreT<ST>;
    using T = typename S::CT;
    constexpr int Q = L::Q;
    const long long plane = P.plane;
    const int idx = y * P.pitch + x;
    T h[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = S::ld(A + i * plane + idx);
    Coef<T> C;
    double Fx = 0.0, Fy = 0.0;  // no fix-up on this step: stays zero
    prepare<L, ST, COLL, 0, OWN_NONE>(P, A, x, y, cls, P.dv, P.dv_f, h, Fx, Fy, C);
    // output i goes to plane opp(i)
    emit_outputs<L, ST, COLL>(C, h, [&](int i, T v) { S::st(A + opp_of<L>(i) * plane + idx, v); });
}

// One launch = one step; PHASE 0 the even (pull-push) step, 1 the odd (local) one.  P.dst is the
// single buffer; force_out[0] and force_out[1] get the forces of steps n and n + 1 (PHASE 0 only).
template <class L, class ST, int COLL, int PHASE>
__global__ void __launch_bounds__(512) step_kernel_aa(const __grid_constant__ InstDev P) {
    pdl_wait_then_release();
    const int tile = blockIdx.x;
    const int slot = P.tile_slot[tile];
    const int tx = tile % P.ntx, ty = tile / P.ntx;
    const int x = tx * blockDim.x + threadIdx.x;
    const int y = ty * blockDim.y + threadIdx.y;
    const int cls = (x < P.nx && y < P.ny) ? (int)P.cls[y * P.pitch + x] : (int)NODE_SOLID;
    ST* A = static_cast<ST*>(P.dst);
    if (PHASE == 0) {
        double F[4] = {0.0, 0.0, 0.0, 0.0};
        if (cls != NODE_SOLID) aa_pull_push<L, ST, COLL>(P, A, x, y, cls, F[0], F[1], F[2], F[3]);
        tile_epilogue_n<2>(P, slot, P.force_out, F);
    } else if (cls != NODE_SOLID) {
        aa_local<L, ST, COLL>(P, A, x, y, cls);
    }
}

template <class L, class ST, int COLL, int PHASE>
cudaError_t launch_step_aa(const InstDev& P, dim3 block, cudaStream_t stream) {
    return launch_pdl(step_kernel_aa<L, ST, COLL, PHASE>, dim3(P.ntiles), block, 0, stream, P);
}

// Launcher of the in-place step for (lattice Q, storage, collision, phase); nullptr if not built.
StepLaunchFn find_aa_launcher(int Q, int storage, int coll, int phase);

}  // namespace lbm
