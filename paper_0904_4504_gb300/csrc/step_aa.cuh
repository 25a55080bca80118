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

// h_i = A[x - c_i][opp(i)], periodic in x and y.
template <class L, class ST>
__device__ __forceinline__ void gather_swapped(const InstDev& P, const ST* src, int x, int y,
                                               typename StoreT<ST>::CT (&h)[L::Q]) {
    using S = StoreT<ST>;
    constexpr int Q = L::Q, R = L::R;
    const long long plane = P.plane;
    int roff[2 * R + 1], col[2 * R + 1];
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
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of<L>(i), cy = cy_of<L>(i);
        h[i] = S::ld(src + opp_of<L>(i) * plane + roff[cy + R] + col[cx + R]);
    }
}

// Even step of one node: pull (swapped), wall fix-up, collide, push.  (Fx, Fy) gets the force of
// step n, (Gx, Gy) the force of step n + 1 from the links bounced on the push.
template <class L, class ST, int COLL>
__device__ __forceinline__ void aa_pull_push(const InstDev& P, ST* A, int x, int y, int cls, double& Fx,
                                             double& Fy, double& Gx, double& Gy) {
    using S = StoreT<ST>;
    using T = typename S::CT;
    constexpr int Q = L::Q, R = L::R;
    const long long plane = P.plane;
    const int idx = y * P.pitch + x;
    T h[Q];
    gather_swapped<L, ST>(P, A, x, y, h);
    Coef<T> C;
    prepare<L, ST, COLL, 0, OWN_SWAPPED>(P, A, x, y, cls, P.dv, P.dv_f, h, Fx, Fy, C);

    // push targets: rows and columns of x + c_i, periodic
    int roff[2 * R + 1], col[2 * R + 1];
#pragma unroll
    for (int d = -R; d <= R; ++d) {
        int ys = y + d;
        ys += ys < 0 ? P.ny : 0;
        ys -= ys >= P.ny ? P.ny : 0;
        int xs = x + d;
        xs += xs < 0 ? P.nx : 0;
        xs -= xs >= P.nx ? P.nx : 0;
        roff[d + R] = ys * P.pitch;
        col[d + R] = xs;
    }
    // link x -> x + c_i is blocked exactly when pull link opp(i) of x is
    ulonglong2 lk = make_ulonglong2(0ull, 0ull);
    if (cls == NODE_BOUNDARY) lk = P.links[idx];
    const unsigned long long blk = lk.x | lk.y;
    const bool off = sizeof(ST) == 2 && P.stream_off;

    auto push = [&](int i, T o) {
        const int j = opp_of<L>(i);
        if ((blk >> j) & 1ull) {
            // comes back as direction j at x in step n + 1 (Eq. 12 with U_w of step n + 1)
            double mw = 0.0;
            if ((lk.x >> j) & 1ull) {
                if (P.moving) mw = P.mw_k * cx_of<L>(j) * P.dv2;
                // the value the two-buffer step would read back: o rounded to the storage type
                const T own = S::rnd(o - (off ? (T)P.Hs[i] : (T)0)) + (off ? (T)P.Hs[i] : (T)0);
                const double hs = 2.0 * (double)own + mw;
                const double ws = w_of<L>(j) * P.s;
                Gx -= cx_of<L>(j) * ws * hs;
                Gy -= cy_of<L>(j) * ws * hs;
            }
            S::st(A + j * plane + idx, o + (T)mw - (off ? (T)P.Hs[j] : (T)0));
        } else {
            S::st(A + i * plane + roff[cy_of<L>(i) + R] + col[cx_of<L>(i) + R], o - (off ? (T)P.Hs[i] : (T)0));
        }
    };
    S::st(A + idx, eval_rest<L, COLL, T>(C, h[0]) - (off ? (T)P.Hs[0] : (T)0));
#pragma unroll
    for (int k = 0; k < L::NP; ++k) {
        T op, omn;
        eval_pair<L, COLL, T>(C, k, h[1 + 2 * k], h[2 + 2 * k], op, omn);
        push(1 + 2 * k, op);
        push(2 + 2 * k, omn);
    }
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
    const bool off = sizeof(ST) == 2 && P.stream_off;
    S::st(A + idx, eval_rest<L, COLL, T>(C, h[0]) - (off ? (T)P.Hs[0] : (T)0));
#pragma unroll
    for (int k = 0; k < L::NP; ++k) {
        T op, omn;
        eval_pair<L, COLL, T>(C, k, h[1 + 2 * k], h[2 + 2 * k], op, omn);
        S::st(A + (2 + 2 * k) * plane + idx, op - (off ? (T)P.Hs[1 + 2 * k] : (T)0));
        S::st(A + (1 + 2 * k) * plane + idx, omn - (off ? (T)P.Hs[2 + 2 * k] : (T)0));
    }
}

// One launch = one step; PHASE 0 the even (pull-push) step, 1 the odd (local) one.  P.dst is the
// single buffer; force_out[0] and force_out[1] get the forces of steps n and n + 1 (PHASE 0 only).
template <class L, class ST, int COLL, int PHASE>
__global__ void __launch_bounds__(512) step_kernel_aa(const __grid_constant__ InstDev P) {
    const int tile = blockIdx.x;
    const int tx = tile % P.ntx, ty = tile / P.ntx;
    const int x = tx * blockDim.x + threadIdx.x;
    const int y = ty * blockDim.y + threadIdx.y;
    const int cls = (x < P.nx && y < P.ny) ? (int)P.cls[y * P.pitch + x] : (int)NODE_SOLID;
    ST* A = static_cast<ST*>(P.dst);
    if (PHASE == 0) {
        double F[4] = {0.0, 0.0, 0.0, 0.0};
        if (cls != NODE_SOLID) aa_pull_push<L, ST, COLL>(P, A, x, y, cls, F[0], F[1], F[2], F[3]);
        tile_epilogue_n<2>(P, tile, P.force_out, F);
    } else if (cls != NODE_SOLID) {
        aa_local<L, ST, COLL>(P, A, x, y, cls);
    }
}

template <class L, class ST, int COLL, int PHASE>
cudaError_t launch_step_aa(const InstDev& P, dim3 block, cudaStream_t stream) {
    step_kernel_aa<L, ST, COLL, PHASE><<<P.ntiles, block, 0, stream>>>(P);
    return cudaGetLastError();
}

// Launcher of the in-place step for (lattice Q, storage, collision, phase); nullptr if not built.
StepLaunchFn find_aa_launcher(int Q, int storage, int coll, int phase);

}  // namespace lbm
