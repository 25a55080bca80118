// step_q9v.cuh -- the D2Q9 step with 16-bit storage, four neighbouring nodes per thread.
//
// With nine populations per node the D2Q9 step does little arithmetic per byte, so the one-node-
// per-thread kernels spend most of their instructions on addressing, per-element loads, stores and
// conversions and are bound by instruction issue, not by HBM.  Here each thread owns four
// x-neighbouring nodes (x0 .. x0 + 3, x0 a multiple of 4, so 8-byte aligned in every row of every
// plane): per direction it loads the four stored values of its source row with one 8-byte load,
// takes the value shifted in by c_x = +1 or -1 from the neighbouring lane (warp shuffle) or, at a
// warp's ends and the periodic seam, with one 2-byte load, applies the wall rule node by node
// (bb_fixup, Eq. 12, with the force), evaluates the collision of two nodes per packed FP32
// instruction (q9_collide2: Eqs. 14-19, the expressions of coef_tail / eval_pair), and stores the
// four outputs of each direction with one 8-byte store.  A warp covers 128 nodes of one row, a block
// 128 x 4.  The last vector of a row that does not end on a multiple of 4 takes the per-node path.
#pragma once

#include "step_kernel.cuh"

namespace lbm {

template <class ST> struct Half16;
template <> struct Half16<__half> {
    static __device__ __forceinline__ float lo(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }
    static __device__ __forceinline__ float hi(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }
    static __device__ __forceinline__ unsigned pack(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const unsigned*>(&h);
    }
};
template <> struct Half16<__nv_bfloat16> {
    static __device__ __forceinline__ float lo(unsigned w) { return __uint_as_float(w << 16); }
    static __device__ __forceinline__ float hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }
    static __device__ __forceinline__ unsigned pack(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const unsigned*>(&h);
    }
};

// F2 with both lanes c.
__device__ __forceinline__ F2 bc2(float c) { return f2(c, c); }

// The D2Q9 collision of two nodes at once, one per lane of the packed FP32 operations: moments
// (Eq. 16) of the pulled and wall-fixed populations H (storage units, relative to the stream offset
// for the regularized collision, absolute for BGK, as prepare leaves them), the equilibrium
// (Eq. 15), then the regularized collision (Eqs. 18-19) or plain BGK, with the body-force source and
// the storage scale; OUT receives the nine outputs in storage units (relative to the stream offset
// of the stored state).  The same expressions as coef_tail / eval_pair, written for D2Q9 (second-
// order equilibrium) with both nodes in one instruction.
template <int COLL>
__device__ __forceinline__ void q9_collide2(const InstDev& P, float dv_f, const F2 (&H)[9], F2 (&OUT)[9]) {
    constexpr float w0 = 4.f / 9.f, w1 = 1.f / 9.f, w2 = 1.f / 36.f, th = 1.f / 3.f;
    // Eq. 16 by velocity group: (1,0), (0,1) pair by pair, (1,1) and (1,-1) together
    const F2 sp0 = add2(H[1], H[2]), dm0 = sub2(H[1], H[2]);
    const F2 sp1 = add2(H[3], H[4]), dm1 = sub2(H[3], H[4]);
    const F2 sp2 = add2(H[5], H[6]), dm2 = sub2(H[5], H[6]);
    const F2 sp3 = add2(H[7], H[8]), dm3 = sub2(H[7], H[8]);
    const F2 S = add2(sp2, sp3), D = sub2(sp2, sp3), Jp = add2(dm2, dm3), Jm = sub2(dm2, dm3);
    const F2 W1 = bc2(w1), W2 = bc2(w2);
    F2 m0 = fma2(W2, S, fma2(W1, add2(sp0, sp1), mul2(bc2(w0), H[0])));
    F2 jx = fma2(W2, Jp, mul2(W1, dm0));
    F2 jy = fma2(W2, Jm, mul2(W1, dm1));
    F2 pxx = fma2(W2, S, mul2(W1, sp0));
    F2 pxy = mul2(W2, D);
    F2 pyy = fma2(W2, S, mul2(W1, sp1));
    if (COLL == COLL_REG && P.stream_off) {
        m0 = add2(m0, bc2(P.HM[0])); jx = add2(jx, bc2(P.HM[1])); jy = add2(jy, bc2(P.HM[2]));
        pxx = add2(pxx, bc2(P.HM[3])); pxy = add2(pxy, bc2(P.HM[4])); pyy = add2(pyy, bc2(P.HM[5]));
    }
    const F2 sc = bc2(P.s_f);
    m0 = mul2(m0, sc); jx = mul2(jx, sc); jy = mul2(jy, sc);
    pxx = mul2(pxx, sc); pxy = mul2(pxy, sc); pyy = mul2(pyy, sc);
    // Eq. 15 and the source, in physical units
    const F2 rho = add2(bc2(P.rho0_f), m0);
    float r0, r1;
    f2_split(rho, r0, r1);
    const F2 irho = f2(__frcp_rn(r0), __frcp_rn(r1));
    const F2 Fbx = P.body_force ? mul2(rho, bc2(dv_f)) : bc2(0.f);
    const F2 half = bc2(0.5f), three = bc2(3.f);
    const F2 ux = mul2(fma2(half, Fbx, jx), irho);
    const F2 uy = mul2(jy, irho);
    const F2 ax = mul2(ux, three), ay = mul2(uy, three);
    const F2 b = mul2(fma2(uy, uy, mul2(ux, ux)), three);
    const F2 hrho = mul2(half, rho);
    F2 e0 = sub2(m0, mul2(hrho, b));
    F2 e1 = hrho, o0 = rho;
    F2 kf = mul2(bc2(P.src_k_f), Fbx);
    F2 kfu = mul2(sub2(bc2(0.f), kf), ux);
    const F2 is = bc2(P.inv_s_f);
    F2 cbase, obase;
    F2 rxx, rxy, ryy, om;
    if (COLL == COLL_REG) {
        // Eq. 19: Pi^ne = Pi - rho theta I - rho u u
        const F2 Th = bc2(th);
        const F2 Pxx = sub2(sub2(pxx, mul2(m0, Th)), mul2(mul2(rho, ux), ux));
        const F2 Pxy = sub2(pxy, mul2(mul2(rho, ux), uy));
        const F2 Pyy = sub2(sub2(pyy, mul2(m0, Th)), mul2(mul2(rho, uy), uy));
        const F2 A = bc2(P.reg_a_f);
        rxx = mul2(mul2(A, Pxx), is);
        rxy = mul2(mul2(bc2(2.f), mul2(A, Pxy)), is);
        ryy = mul2(mul2(A, Pyy), is);
        cbase = mul2(add2(sub2(e0, mul2(mul2(A, Th), add2(Pxx, Pyy))), kfu), is);
        obase = mul2(mul2(mul2(half, Fbx), three), is);   // kept J^ne = -F/2 plus the source
        om = bc2(0.f);
    } else {
        rxx = rxy = ryy = bc2(0.f);
        om = bc2(P.omega_c_f);
        e0 = mul2(e0, is);
        cbase = mul2(kfu, is);
        obase = mul2(kf, is);
    }
    e1 = mul2(e1, is);
    o0 = mul2(o0, is);
    kf = mul2(kf, is);
    // constant parts per m = |c_x| (0, 1), less the stream offset of the stored state
    const F2 ce0 = sub2(cbase, bc2(P.He[0])), ce1 = sub2(cbase, bc2(P.He[1]));
    const F2 co0 = sub2(bc2(0.f), bc2(P.Ho[0])), co1 = sub2(obase, bc2(P.Ho[1]));
    // pairs (1,0), (0,1), (1,1), (1,-1): a = c.u / theta
    const F2 aa[4] = {ax, ay, add2(ax, ay), sub2(ax, ay)};
    if (COLL == COLL_REG) {
        OUT[0] = ce0;
        const F2 rsum = add2(rxx, ryy);
        const F2 q[4] = {add2(ce1, rxx), add2(ce0, ryy), add2(add2(ce1, rsum), rxy), sub2(add2(ce1, rsum), rxy)};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const F2 a = aa[k];
            const F2 a2 = mul2(a, a);
            F2 E = fma2(a2, e1, q[k]);
            if (k != 1) E = fma2(a, kf, E);   // px kf, px = 1 except for (0,1)
            const F2 O = fma2(a, o0, k == 1 ? co0 : co1);
            OUT[1 + 2 * k] = add2(E, O);
            OUT[2 + 2 * k] = sub2(E, O);
        }
    } else {
        OUT[0] = add2(fma2(om, sub2(e0, H[0]), H[0]), ce0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const F2 a = aa[k];
            const F2 a2 = mul2(a, a);
            const F2 E = fma2(a2, e1, e0);
            const F2 O = mul2(a, o0);
            const F2 Es = k == 1 ? ce0 : fma2(a, kf, ce1);
            const F2 Os = k == 1 ? co0 : co1;
            const F2 hp = H[1 + 2 * k], hm = H[2 + 2 * k];
            OUT[1 + 2 * k] = add2(fma2(om, sub2(add2(E, O), hp), hp), add2(Es, Os));
            OUT[2 + 2 * k] = add2(fma2(om, sub2(sub2(E, O), hm), hm), sub2(Es, Os));
        }
    }
}

// The source rows of one thread's four nodes: per direction the four stored values of its pulled
// row (w0: elements 0, 1; w1: elements 2, 3) and the value shifted in by c_x (h(x0 - 1) for
// c_x = +1, h(x0 + 4) for c_x = -1).
struct Q9Row {
    unsigned w0[9], w1[9];
    unsigned short sh[9];
};

// Loads of the row y of a thread's nodes x0 .. x0 + 3 (warp-uniform y: the shuffles need the whole
// warp; `any`: this thread owns a node inside the grid).
template <class ST>
__device__ __forceinline__ void q9v_load(const InstDev& P, int x0, int y, int lane, bool any, Q9Row& R) {
    using L = D2Q9;
    const ST* __restrict__ src = static_cast<const ST*>(P.src);
    const unsigned plane = (unsigned)P.plane;
    const int nx = P.nx, ny = P.ny, pitch = P.pitch;
    int ys[3];  // source row of c_y = -1, 0, +1
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
        int r = y - d;
        r += r < 0 ? ny : 0;
        r -= r >= ny ? ny : 0;
        ys[d + 1] = r;
    }
    const int xl = x0 == 0 ? nx - 1 : x0 - 1;   // left neighbour column (periodic)
    const int xr = x0 + 4 >= nx ? x0 + 4 - nx : x0 + 4;
    const bool edge_l = lane == 0 || x0 == 0;
    const bool edge_r = lane == 31 || x0 + 4 >= nx;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = cx_of<L>(i), cy = cy_of<L>(i);
        const unsigned rowoff = (unsigned)(i * plane + ys[cy + 1] * pitch);
        uint2 v = make_uint2(0u, 0u);
        if (any) v = *reinterpret_cast<const uint2*>(src + rowoff + x0);
        R.w0[i] = v.x;
        R.w1[i] = v.y;
        if (cx == 1) {
            const unsigned up = __shfl_up_sync(0xffffffffu, v.y, 1);
            unsigned short s = (unsigned short)(up >> 16);
            if (edge_l && any) s = *reinterpret_cast<const unsigned short*>(src + rowoff + xl);
            R.sh[i] = s;
        } else if (cx == -1) {
            const unsigned dn = __shfl_down_sync(0xffffffffu, v.x, 1);
            unsigned short s = (unsigned short)(dn & 0xffffu);
            if (edge_r && any && x0 + 4 <= nx) s = *reinterpret_cast<const unsigned short*>(src + rowoff + xr);
            R.sh[i] = s;
        } else {
            R.sh[i] = 0;
        }
    }
}

// Collision and store of a thread's four nodes of row y from their loaded source rows.
template <class ST, int COLL>
__device__ __forceinline__ void q9v_compute(const InstDev& P, int x0, int y, unsigned cls4, const Q9Row& R, double& Fx,
                                            double& Fy) {
    using L = D2Q9;
    using H = Half16<ST>;
    constexpr int Q = 9;
    const ST* __restrict__ src = static_cast<const ST*>(P.src);
    const unsigned plane = (unsigned)P.plane;
    const int nx = P.nx, pitch = P.pitch;
    ST* __restrict__ dst = static_cast<ST*>(P.dst) + (size_t)y * pitch + x0;
    unsigned o0[Q], o1[Q];
    if (x0 + 4 <= nx) {
        // value of direction i pulled to node j (0..3) of this thread
        auto pulled = [&](int i, int j) -> float {
            const int cx = cx_of<L>(i);
            const int e = j - cx;  // element of the loaded vector, -1 or 4: the shifted-in one
            if (e < 0 || e > 3) return H::lo((unsigned)R.sh[i]);
            return e == 0 ? H::lo(R.w0[i]) : e == 1 ? H::hi(R.w0[i]) : e == 2 ? H::lo(R.w1[i]) : H::hi(R.w1[i]);
        };
        const bool off = P.stream_off != 0;
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
            const int ca = (cls4 >> (16 * pr)) & 0xff, cb = (cls4 >> (16 * pr + 8)) & 0xff;
            if (ca == NODE_SOLID && cb == NODE_SOLID) {
#pragma unroll
                for (int i = 0; i < Q; ++i) (pr == 0 ? o0 : o1)[i] = 0u;
                continue;
            }
            // pulled populations of the pair's two nodes; the stream offset and the wall rule
            // (Eq. 12, with the momentum handed to the body) per node, as in prepare
            float ha[Q], hb[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                ha[i] = pulled(i, 2 * pr);
                hb[i] = pulled(i, 2 * pr + 1);
                if (off && COLL == COLL_BGK) {
                    ha[i] += off_l<L>(P, i);
                    hb[i] += off_l<L>(P, i);
                }
            }
            const int idx = y * pitch + x0 + 2 * pr;
            if (ca == NODE_BOUNDARY) bb_fixup<L, ST, COLL, OWN_OPP>(P, src, idx, P.dv, ha, Fx, Fy);
            if (cb == NODE_BOUNDARY) bb_fixup<L, ST, COLL, OWN_OPP>(P, src, idx + 1, P.dv, hb, Fx, Fy);
            F2 Hp[Q], Op[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) Hp[i] = f2(ha[i], hb[i]);
            q9_collide2<COLL>(P, P.dv_f, Hp, Op);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float va, vb;
                f2_split(Op[i], va, vb);
                (pr == 0 ? o0 : o1)[i] = H::pack(ca == NODE_SOLID ? 0.f : va, cb == NODE_SOLID ? 0.f : vb);
            }
        }
    } else {
        // the last vector of a row that ends inside it: per-node gathers with the periodic wrap
#pragma unroll 1
        for (int pr = 0; pr < 2; ++pr) {
            float out[2][Q];
            for (int jj = 0; jj < 2; ++jj) {
                const int j = 2 * pr + jj;
                const int c = (cls4 >> (8 * j)) & 0xff;
                if (x0 + j >= nx || c == NODE_SOLID) {
#pragma unroll
                    for (int i = 0; i < Q; ++i) out[jj][i] = 0.f;
                    continue;
                }
                float h[Q];
                gather_global<L, ST>(P, src, x0 + j, y, h);
                Coef<float> C;
                prepare<L, ST, COLL>(P, P.src, x0 + j, y, c, P.dv, P.dv_f, h, Fx, Fy, C);
                emit_outputs<L, ST, COLL>(C, h, [&](int i, float v) { out[jj][i] = v; });
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) (pr == 0 ? o0 : o1)[i] = H::pack(out[0][i], out[1][i]);
        }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) *reinterpret_cast<uint2*>(dst + (size_t)i * plane) = make_uint2(o0[i], o1[i]);
}

// NR rows per thread, 4 apart (tiles of 128 x 4 NR nodes): the loads of all NR rows are issued
// before the first row is computed, so that more bytes are in flight per thread.
template <class ST, int COLL, int NR, int MINB>
__global__ void __launch_bounds__(128, MINB) step_kernel_q9v(const __grid_constant__ InstDev P) {
    const int t = blockIdx.x;
    const int slot = P.tile_slot[t];  // geometry (host-written): read before the wait
    const int lane = threadIdx.x;
    const int x0 = (t % P.ntx) * 128 + 4 * lane;
    const int y0 = (t / P.ntx) * (4 * NR) + threadIdx.y;
    unsigned cls4[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int y = y0 + 4 * r;
        cls4[r] = 0x01010101u;  // NODE_SOLID x 4
        if (y < P.ny && x0 < P.nx) cls4[r] = *reinterpret_cast<const unsigned*>(P.cls + (size_t)y * P.pitch + x0);
    }
    pdl_wait_then_release();
    double Fx = 0.0, Fy = 0.0;
    Q9Row R[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int y = y0 + 4 * r;
        if (y < P.ny) q9v_load<ST>(P, x0, y, lane, x0 < P.nx, R[r]);  // warp-uniform row test
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int y = y0 + 4 * r;
        if (y < P.ny && x0 < P.nx) q9v_compute<ST, COLL>(P, x0, y, cls4[r], R[r], Fx, Fy);
    }
    tile_epilogue(P, slot, P.force_out, Fx, Fy);
}

template <class ST, int COLL, int NR, int MINB>
cudaError_t launch_step_q9v(const InstDev& P, dim3, cudaStream_t stream) {
    return launch_pdl(step_kernel_q9v<ST, COLL, NR, MINB>, dim3(P.ntiles), dim3(32, 4), 0, stream, P);
}

}  // namespace lbm
