// step_kernel.cuh -- the fused LBGK time step on sm_103a.
//
// One launch performs, for every fluid node of one or more lattices (Sec. 5 of the paper, in its
// order): advection by pull (Eq. 17) with bounce-back on blocked links (Eq. 12), the moments
// (Eq. 16), the Hermite equilibrium (Eq. 15 or its 4th-order continuation), the regularized
// collision (Eqs. 18-19) or the plain BGK step (Eq. 14), an optional body force, and the store.
// The momentum given to the body by bounce-back is reduced in FP64 (warp shuffles, then a fixed
// slot per tile that holds body links); the last of those tiles to finish sums the slots in a
// fixed order and writes (Fx, Fy) of the step.  Tiles without body links skip the reduction
// entirely.  No block ever waits for another.
//
// Storage.  Populations are kept as scaled deviations from the rest state,
//     h_i = (f_i - w_i rho0) / (w_i s),
// structure-of-arrays [Q][ny][pitch].  s = 1 for FP64/FP32 storage and s = u0 (the drive
// amplitude) for BF16/FP16, so that every direction is O(1) and far from the 16-bit subnormal
// range.  The weights cancel out of the equilibrium and collision in these units.  Arithmetic is
// FP64 for FP64 storage and FP32 otherwise; the wall force is always accumulated in FP64.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "lattice.cuh"

namespace lbm {

enum Storage { ST_F64 = 0, ST_F32 = 1, ST_BF16 = 2, ST_F16 = 3 };
enum Collision { COLL_BGK = 0, COLL_REG = 1 };

// Node classes of the `cls` array.
enum NodeClass : uint8_t { NODE_BULK = 0, NODE_SOLID = 1, NODE_BOUNDARY = 2 };

// Everything one launch needs to know about one lattice instance.
struct InstDev {
    const void* src;             // h at step n, [Q][ny][pitch]
    void* dst;                   // h at step n+1
    const uint8_t* cls;          // [ny][pitch] NodeClass
    const ulonglong2* links;     // [ny][pitch]: .x bit i = link i blocked by the body (label 1),
                                 //              .y bit i = blocked by a static wall (label 2)
    const int* tile_slot;        // [ntiles] force-partial slot of a tile, -1 if it has no body link
    double2* partials;           // [nslots] per-tile FP64 force partials (scratch)
    unsigned int* ticket;        // slot tiles of the current step that have finished (scratch, 0
                                 // between launches: the last slot tile resets it)
    double2* force_out;          // force on the body during this step (written by the last slot tile)
    int* err;                    // bit 0: non-finite force seen
    double dv;                   // drive of this step: U_w(n + 1/2) (wall) or g(n + 1/2) (body force)
    double dv2;                  // drive of the next step, n + 3/2 (in-place AA streaming only)
    double2 fconst;              // geometry-only part of the force, -sum c_i 2 w_i rho0
    long long plane;             // ny * pitch
    int nx, ny, pitch;
    int ntx;                     // tiles along x
    int ntiles, nslots;
    int eq_order;                // 2 or 4
    int moving;                  // 1: body links carry the moving-wall term (wall drive)
    int wall_ds;                 // 0: bounce-back (Eq. 12); 1: diffuse scattering (Eq. 11)
    int body_force;              // 1: fluid gets rho * g (body-frame drive)
    double rho0;
    double s, inv_s;             // storage scale
    double omega_c;              // 1/tau
    double reg_a;                // (1 - 1/tau) / (2 theta^2)
    double src_k;                // (1 - 1/(2 tau)) / theta
    double mw_k;                 // 2 rho0 / (theta s): moving-wall term per unit c_i.U_w
    // FP32 copies of the constants above (and of dv), so that FP32 arithmetic converts nothing per
    // node: double -> float conversions run on the FP64 pipe, which is slow on this GPU
    float dv_f, rho0_f, s_f, inv_s_f, omega_c_f, reg_a_f, src_k_f, dv2_f;
    // 16-bit body-frame runs store h_i - H_i(n), with H_i(n) the (scaled) equilibrium deviation of
    // the uniform stream U(n) = sum_{k<n} g(k + 1/2) that the body force sets up; far from the body
    // the stored values are then small and so are their rounding errors.  The stream is along x, so
    // H_i depends on c_ix only: Hl (the state read) and Hs (the state written) hold it for
    // c_ix = -3..3 at index c_ix + 3.  HM: moments sum_i w_i {1, c, cc} H_i of Hl (scaled units).
    // He, Ho: the even and odd parts of Hs in c_x, He[m] = (Hs(m) + Hs(-m)) / 2 and
    // Ho[m] = (Hs(m) - Hs(-m)) / 2 for m = |c_x|; the collision folds them into its per-node
    // coefficients, so outputs leave it already relative to the stream.  All zero when stream_off
    // is clear.
    int stream_off;
    float HM[6];
    float Hl[7];
    float Hs[7];
    float He[4];
    float Ho[4];
};

// Programmatic dependent launch.  Step kernels are launched so that the next kernel of the stream
// may be scheduled while this one drains: every step kernel first waits for the previous grid of
// its stream to complete (its outputs are this step's inputs, including the force scratch), then
// lets the next one launch.  The next grid is launched only after every block of this one has
// passed that point, so its blocks never take SM slots that this grid still needs.
__device__ __forceinline__ void pdl_wait_then_release() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch a step kernel with programmatic stream serialization (disabled when the environment
// sets LBM_PDL=0: plain stream order).
bool pdl_enabled();

template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Stream-offset constants of direction i (see InstDev): read / written state.
template <class L>
__device__ __forceinline__ float off_l(const InstDev& P, int i) { return P.Hl[cx_of<L>(i) + 3]; }
template <class L>
__device__ __forceinline__ float off_s(const InstDev& P, int i) { return P.Hs[cx_of<L>(i) + 3]; }

// A launch constant in the arithmetic type T: the double itself, or its FP32 copy.
template <class T>
__device__ __forceinline__ T kconst(double d, float f);
template <>
__device__ __forceinline__ double kconst<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float kconst<float>(double, float f) { return f; }

template <class ST> struct StoreT;
// Loads and stores of the storage type; ld2/st2 move two neighbouring values (p aligned to two
// elements) with one access; rnd(v) is v rounded to the storage type (what a store and a load give).
// st stores through a generic pointer (global or shared memory); stg stores to global memory only,
// for 16-bit storage as a streaming store (st.global.cs): the next step reads the populations back
// long after they have left L2, and marking them first to evict keeps the staged loads' shared halo
// sectors in L2 longer.
// ldc is a plain weak load (ld.global.ca), never the read-only path (ld.global.nc) that the
// compiler may pick for a const __restrict__ pointer: the persistent batch kernel reads populations
// that other blocks of the same launch wrote.  They are visible to weak loads that follow the
// acquire of their producer's release (in the block, through the block barrier), which is what the
// memory model guarantees; it guarantees nothing for the read-only path.
template <> struct StoreT<double> {
    using CT = double;
    static __device__ __forceinline__ double rnd(double v) { return v; }
    static __device__ __forceinline__ double ld(const double* p) { return *p; }
    static __device__ __forceinline__ double ldc(const double* p) {
        double v;
        asm volatile("ld.global.ca.f64 %0, [%1];" : "=d"(v) : "l"(p));
        return v;
    }
    static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
    static __device__ __forceinline__ void stg(double* p, double v) { *p = v; }
    static __device__ __forceinline__ void ld2(const double* p, double& a, double& b) {
        const double2 v = *reinterpret_cast<const double2*>(p);
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void st2(double* p, double a, double b) {
        *reinterpret_cast<double2*>(p) = make_double2(a, b);
    }
};
template <> struct StoreT<float> {
    using CT = float;
    static __device__ __forceinline__ float rnd(float v) { return v; }
    static __device__ __forceinline__ float ld(const float* p) { return *p; }
    static __device__ __forceinline__ float ldc(const float* p) {
        float v;
        asm volatile("ld.global.ca.f32 %0, [%1];" : "=f"(v) : "l"(p));
        return v;
    }
    static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
    static __device__ __forceinline__ void stg(float* p, float v) { *p = v; }
    static __device__ __forceinline__ void ld2(const float* p, float& a, float& b) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void st2(float* p, float a, float b) {
        *reinterpret_cast<float2*>(p) = make_float2(a, b);
    }
};
template <> struct StoreT<__nv_bfloat16> {
    using CT = float;
    static __device__ __forceinline__ float rnd(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ float ldc(const __nv_bfloat16* p) {
        unsigned short v;
        asm volatile("ld.global.ca.u16 %0, [%1];" : "=h"(v) : "l"(p));
        return __bfloat162float(__ushort_as_bfloat16(v));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ void stg(__nv_bfloat16* p, float v) {
        asm("st.global.cs.b16 [%0], %1;" ::"l"(p), "h"(__bfloat16_as_ushort(__float2bfloat16_rn(v))));
    }
    static __device__ __forceinline__ void ld2(const __nv_bfloat16* p, float& a, float& b) {
        const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void st2(__nv_bfloat16* p, float a, float b) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
    }
};
template <> struct StoreT<__half> {
    using CT = float;
    static __device__ __forceinline__ float rnd(float v) { return __half2float(__float2half_rn(v)); }
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ float ldc(const __half* p) {
        unsigned short v;
        asm volatile("ld.global.ca.u16 %0, [%1];" : "=h"(v) : "l"(p));
        return __half2float(__ushort_as_half(v));
    }
    static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ void stg(__half* p, float v) {
        asm("st.global.cs.b16 [%0], %1;" ::"l"(p), "h"(__half_as_ushort(__float2half_rn(v))));
    }
    static __device__ __forceinline__ void ld2(const __half* p, float& a, float& b) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void st2(__half* p, float a, float b) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
    }
};

// Eq. 17 from global memory: h_i^adv(x) = h_i(x - c_i), periodic in x and y.
template <class L, class ST, bool COH = false>
__device__ __forceinline__ void gather_global(const InstDev& P, const ST* __restrict__ src, int x, int y,
                                              typename StoreT<ST>::CT (&h)[L::Q]) {
    using S = StoreT<ST>;
    constexpr int Q = L::Q, R = L::R;
    const unsigned plane = (unsigned)P.plane;  // Q * plane < 2^32 (checked at creation)
    unsigned roff[2 * R + 1], col[2 * R + 1];
#pragma unroll
    for (int d = -R; d <= R; ++d) {
        int ys = y - d;
        ys += ys < 0 ? P.ny : 0;
        ys -= ys >= P.ny ? P.ny : 0;
        int xs = x - d;
        xs += xs < 0 ? P.nx : 0;
        xs -= xs >= P.nx ? P.nx : 0;
        roff[d + R] = (unsigned)(ys * P.pitch);
        col[d + R] = (unsigned)xs;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of<L>(i), cy = cy_of<L>(i);
        // 32-bit element offset, widened once: one multiply-add per address
        const ST* p = src + (unsigned)(i * plane + roff[cy + R] + col[cx + R]);
        h[i] = COH ? S::ldc(p) : S::ld(p);
    }
}

// Per-node coefficients of the collision output: every output is a polynomial in a = c_i.u/theta
// whose coefficients depend on the node only.
template <class T>
struct Coef {
    T ax, ay;                  // u / theta
    T c0, e1, e2, o0, o1;      // even part c0 + a^2 (e1 + a^2 e2), odd part a (o0 + o1 a^2)
    T rxx, rxy, ryy, hf;       // regularized part and first-order force part
    T kf;                      // force coefficient
    T om, e0, kfu;             // plain BGK: 1/tau, equilibrium constant, even source constant
    // per m = |c_x| (0..3), with the stream offset of the stored state folded in (16-bit storage):
    // regularized: c0 - He[m] and m hf - Ho[m]; plain BGK: kfu - He[m] and m kf - Ho[m]
    T ce[4], co[4];
};

// Bounce-back (fix-up of h on blocked links), moments and collision coefficients of the fluid node
// (x, y) whose pulled populations are in h.  Adds the momentum the node's blocked body links hand
// to the body to (Fx, Fy).  OWN says where the node's own post-collision population opposite to
// link i is: plane opp(i) of src (two buffers, OWN_OPP), plane i (in-place AA streaming, whose
// even steps store directions swapped, OWN_SWAPPED), or nowhere because the wall rules were applied
// when the populations were pushed (OWN_NONE: no fix-up here).
enum OwnPlane { OWN_OPP = 0, OWN_SWAPPED = 1, OWN_NONE = 2 };

// Eq. 16 on deviations: drho = sum g_i, j = sum g_i c_i, Pi' = sum g_i c_i c_i, in the units of
// the populations (w_i divided out).  spdm(k, sp, dm) gives the sum and difference of pair k's two
// populations, h0 the rest population.  The pair tables list pairs in groups of two of one shell:
// (p_x, p_y) and (p_x, -p_y), whose sums S, D and differences Jp, Jm of sp and dm give the six
// moments with one multiply-add each, or (m, 0) and (0, m), taken pair by pair.
template <class L, class T, class SpDm>
__device__ __forceinline__ void moments(SpDm&& spdm, T h0, T& m0, T& jx, T& jy, T& pxx, T& pxy, T& pyy) {
    m0 = (T)L::w0() * h0;
    jx = jy = pxx = pxy = pyy = (T)0;
    auto one = [&](int k, T sp, T dm) {
        const int px = L::px(k), py = L::py(k);
        const double w = L::wp(k);
        m0 += (T)w * sp;
        if (px) jx += (T)(w * px) * dm;
        if (py) jy += (T)(w * py) * dm;
        if (px) pxx += (T)(w * px * px) * sp;
        if (px && py) pxy += (T)(w * px * py) * sp;
        if (py) pyy += (T)(w * py * py) * sp;
    };
#pragma unroll
    for (int k = 0; k < L::NP; k += 2) {
        T sp1, dm1;
        spdm(k, sp1, dm1);
        if (k + 1 == L::NP) {
            one(k, sp1, dm1);
            continue;
        }
        T sp2, dm2;
        spdm(k + 1, sp2, dm2);
        const int px = L::px(k), py = L::py(k);
        if (px && py && L::px(k + 1) == px && L::py(k + 1) == -py && L::wp(k + 1) == L::wp(k)) {
            const double w = L::wp(k);
            const T S = sp1 + sp2, D = sp1 - sp2, Jp = dm1 + dm2, Jm = dm1 - dm2;
            m0 += (T)w * S;
            jx += (T)(w * px) * Jp;
            jy += (T)(w * py) * Jm;
            pxx += (T)(w * px * px) * S;
            pxy += (T)(w * px * py) * D;
            pyy += (T)(w * py * py) * S;
        } else {
            one(k, sp1, dm1);
            one(k + 1, sp2, dm2);
        }
    }
}

// A product rounded on its own (never contracted with a later add into a fused multiply-add).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Collision coefficients of a node from its moments (storage units, relative to the stream offset
// with 16-bit storage and the offset on): Eqs. 15 and 19 and the Guo-type source.  With 16-bit
// storage the moments are scaled by s on the way in and the coefficients by 1/s on the way out.
template <class L, class ST, int COLL>
__device__ __forceinline__ void coef_tail(const InstDev& P, double dv, float dv_f, typename StoreT<ST>::CT m0,
                                          typename StoreT<ST>::CT jx, typename StoreT<ST>::CT jy,
                                          typename StoreT<ST>::CT pxx, typename StoreT<ST>::CT pxy,
                                          typename StoreT<ST>::CT pyy, Coef<typename StoreT<ST>::CT>& C) {
    using T = typename StoreT<ST>::CT;
    constexpr bool SCALED = sizeof(ST) == 2;
    if (SCALED) {
        if (COLL == COLL_REG && P.stream_off) {
            m0 += (T)P.HM[0]; jx += (T)P.HM[1]; jy += (T)P.HM[2];
            pxx += (T)P.HM[3]; pxy += (T)P.HM[4]; pyy += (T)P.HM[5];
        }
        // the storage scale is applied by rounded multiplies that the compiler may not fuse into
        // a later add, so that every kernel variant computes the same bits
        const T s = kconst<T>(P.s, P.s_f);
        m0 = mul_rn(m0, s); jx = mul_rn(jx, s); jy = mul_rn(jy, s);
        pxx = mul_rn(pxx, s); pxy = mul_rn(pxy, s); pyy = mul_rn(pyy, s);
    }
    constexpr double TH = L::theta();
    const T th = (T)TH, ith = (T)(1.0 / TH);
    const T drho = m0;
    const T rho = kconst<T>(P.rho0, P.rho0_f) + drho;
    const T irho = (T)1 / rho;
    const T Fbx = P.body_force ? rho * kconst<T>(dv, dv_f) : (T)0;
    const T ux = (jx + (T)0.5 * Fbx) * irho;
    const T uy = jy * irho;
    C.ax = ux * ith;
    C.ay = uy * ith;
    const T b = (ux * ux + uy * uy) * ith;

    // Eq. 15 (+ 4th order): g_i^eq / w_i = E(a^2) + O(a), a = c_i.u/theta
    T e0 = drho - (T)0.5 * rho * b, e1 = (T)0.5 * rho, e2 = 0, o0 = rho, o1 = 0;
    if (P.eq_order >= 4) {
        e0 += (T)0.125 * rho * b * b;
        e1 -= (T)0.25 * rho * b;
        e2 = rho * (T)(1.0 / 24.0);
        o0 -= (T)0.5 * rho * b;
        o1 = rho * (T)(1.0 / 6.0);
    }
    C.e1 = e1;
    C.e2 = e2;
    C.o0 = o0;
    C.o1 = o1;
    // Guo-type source, even part kf (a c_x - u_x) and odd part c_x * (kf or F/(2 theta))
    const T kf = kconst<T>(P.src_k, P.src_k_f) * Fbx;
    const T kfu = -kf * ux;
    C.kf = kf;
    if (COLL == COLL_REG) {
        // Eq. 19: Pi^ne = Pi - Pi^eq with Pi^eq = rho theta I + rho u u (exact on these lattices)
        const T Pxx = pxx - drho * th - rho * ux * ux;
        const T Pxy = pxy - rho * ux * uy;
        const T Pyy = pyy - drho * th - rho * uy * uy;
        const T A = kconst<T>(P.reg_a, P.reg_a_f);
        C.rxx = A * Pxx;
        C.rxy = (T)2 * A * Pxy;
        C.ryy = A * Pyy;
        C.c0 = e0 - A * th * (Pxx + Pyy) + kfu;
        C.hf = (T)0.5 * Fbx * ith;   // first-order part: kept J^ne = -F/2 plus the source
    } else {
        C.om = kconst<T>(P.omega_c, P.omega_c_f);
        C.e0 = e0;
        C.kfu = kfu;
    }
    if (SCALED) {
        // outputs are wanted in storage units (divided by s): scale the coefficients once per node
        const T is = kconst<T>(P.inv_s, P.inv_s_f);
        C.c0 = mul_rn(C.c0, is); C.e1 = mul_rn(C.e1, is); C.e2 = mul_rn(C.e2, is);
        C.o0 = mul_rn(C.o0, is); C.o1 = mul_rn(C.o1, is);
        C.rxx = mul_rn(C.rxx, is); C.rxy = mul_rn(C.rxy, is); C.ryy = mul_rn(C.ryy, is);
        C.kf = mul_rn(C.kf, is); C.hf = mul_rn(C.hf, is);
        C.e0 = mul_rn(C.e0, is); C.kfu = mul_rn(C.kfu, is);
    }
    // constant parts of the outputs per m = |c_x|; 16-bit storage subtracts the stream offset of
    // the stored state here, once per node (He, Ho are zero when it is off)
    const T cbase = COLL == COLL_REG ? C.c0 : C.kfu, obase = COLL == COLL_REG ? C.hf : C.kf;
#pragma unroll
    for (int m = 0; m <= L::R; ++m) {
        C.ce[m] = SCALED ? cbase - (T)P.He[m] : cbase;
        C.co[m] = SCALED ? (T)m * obase - (T)P.Ho[m] : (T)m * obase;
    }
}

// Eq. 12 on the blocked links of the boundary node at element offset idx: the node's own opposite
// population comes back (from plane opp(i) of src, or plane i with OWN_SWAPPED), plus the moving-wall
// term 2 w_i rho0 c_i.U_w / theta (w_i and s divided out); adds the momentum the node's body links
// hand to the body to (Fx, Fy).  With 16-bit storage and the stream offset on, h holds values
// relative to the stream on entry and exit for the regularized collision, absolute ones for BGK.
template <class L, class ST, int COLL, int OWN, bool COH = false>
__device__ __forceinline__ void bb_fixup(const InstDev& P, const ST* __restrict__ src, int idx, double dv,
                                         typename StoreT<ST>::CT (&h)[L::Q], double& Fx, double& Fy) {
    using S = StoreT<ST>;
    using T = typename S::CT;
    const long long plane = P.plane;
    const bool off = sizeof(ST) == 2 && P.stream_off;
    const ulonglong2 lk = P.links[idx];
    const unsigned long long blk = lk.x | lk.y;
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        if ((blk >> i) & 1ull) {
            const int cx = cx_of<L>(i), cy = cy_of<L>(i);
            const ST* po = src + (OWN == OWN_SWAPPED ? i : opp_of<L>(i)) * plane + idx;
            T own = COH ? S::ldc(po) : S::ld(po);
            if (off) own += (T)off_l<L>(P, opp_of<L>(i));
            double mw = 0.0;
            if ((lk.x >> i) & 1ull) {
                if (P.moving) mw = P.mw_k * cx * dv;
                // momentum c_opp h_opp in, c_i h_i^adv out: -c_i w_i s (h_opp + h_i^adv)
                const double hs = 2.0 * (double)own + mw;
                const double ws = w_of<L>(i) * P.s;
                Fx -= cx * ws * hs;
                Fy -= cy * ws * hs;
            }
            h[i] = own + (T)mw;
            // the regularized path keeps h relative to the stream until the moments
            if (off && COLL == COLL_REG) h[i] -= (T)off_l<L>(P, i);
        }
    }
}

template <class L, class ST, int COLL, int WALL = 0, int OWN = OWN_OPP, bool COH = false>
__device__ __forceinline__ void prepare(const InstDev& P, const void* src_v, int x, int y, int cls, double dv,
                                        float dv_f, typename StoreT<ST>::CT (&h)[L::Q], double& Fx, double& Fy,
                                        Coef<typename StoreT<ST>::CT>& C) {
    using S = StoreT<ST>;
    using T = typename S::CT;
    constexpr int Q = L::Q;
    constexpr bool SCALED = sizeof(ST) == 2;
    const ST* __restrict__ src = static_cast<const ST*>(src_v);
    const long long plane = P.plane;
    const int idx = y * P.pitch + x;

    // stored values relative to the uniform stream: plain BGK needs every h_i, the regularized
    // collision only their moments (HM is added to those below)
    const bool off = SCALED && P.stream_off;
    if (off && COLL == COLL_BGK) {
#pragma unroll
        for (int i = 0; i < Q; ++i) h[i] += (T)off_l<L>(P, i);
    }
    if (cls == NODE_BOUNDARY && WALL == 0 && OWN != OWN_NONE) {
        bb_fixup<L, ST, COLL, OWN, COH>(P, src, idx, dv, h, Fx, Fy);
    } else if (WALL == 1 && cls == NODE_BOUNDARY && OWN == OWN_OPP) {
        // Eq. 11 on blocked links: each wall returns its discrete Maxwellian at the wall velocity,
        // f_i = w_i rho_w (1 + e_i(U_w)), with rho_w set so that the node gets back exactly the mass
        // it sends into that wall (per wall: body = bits of .x, static wall = bits of .y)
        const ulonglong2 lk = P.links[idx];
        const unsigned long long blk = lk.x | lk.y;
        const T rho0 = kconst<T>(P.rho0, P.rho0_f), sT = kconst<T>(P.s, P.s_f);
        const T Ub = P.moving ? kconst<T>(dv, dv_f) : (T)0;
        const T ith = (T)(1.0 / L::theta()), bb = Ub * Ub * ith;
        const bool eq4 = P.eq_order >= 4;
        T in[2] = {0, 0}, mw[2] = {0, 0}, se[2] = {0, 0};
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if ((blk >> i) & 1ull) {
                const int wb = ((lk.x >> i) & 1ull) ? 0 : 1;
                T own = S::ld(src + opp_of<L>(i) * plane + idx);
                if (off) own += (T)off_l<L>(P, opp_of<L>(i));
                h[i] = own;  // kept until the second pass
                const T w = (T)w_of<L>(i);
                in[wb] += w * own;
                mw[wb] += w;
                if (wb == 0) {
                    const T a = (T)cx_of<L>(i) * Ub * ith;
                    T e = a + (T)0.5 * (a * a - bb);
                    if (eq4) e += (a * a * a - (T)3 * a * bb) * (T)(1.0 / 6.0) +
                                  (a * a * a * a - (T)6 * a * a * bb + (T)3 * bb * bb) * (T)(1.0 / 24.0);
                    se[0] += w * e;
                }
            }
        }
        T drw[2], rw[2];  // rho_w - rho0 and rho_w of each wall
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const T den = mw[k] + se[k];
            drw[k] = den > (T)0 ? (sT * in[k] - rho0 * se[k]) / den : (T)0;
            rw[k] = rho0 + drw[k];
        }
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if ((blk >> i) & 1ull) {
                const int cx = cx_of<L>(i), cy = cy_of<L>(i);
                const bool body = (lk.x >> i) & 1ull;
                const int wb = body ? 0 : 1;
                T e = 0;
                if (body) {
                    const T a = (T)cx * Ub * ith;
                    e = a + (T)0.5 * (a * a - bb);
                    if (eq4) e += (a * a * a - (T)3 * a * bb) * (T)(1.0 / 6.0) +
                                  (a * a * a * a - (T)6 * a * a * bb + (T)3 * bb * bb) * (T)(1.0 / 24.0);
                }
                const T hadv = (drw[wb] + rw[wb] * e) / sT;
                if (body) {
                    const double hs = (double)h[i] + (double)hadv;
                    const double ws = w_of<L>(i) * P.s;
                    Fx -= cx * ws * hs;
                    Fy -= cy * ws * hs;
                }
                h[i] = hadv;
                if (off && COLL == COLL_REG) h[i] -= (T)off_l<L>(P, i);
            }
        }
    }

    T m0, jx, jy, pxx, pxy, pyy;
    moments<L, T>([&](int k, T& sp, T& dm) {
        sp = h[1 + 2 * k] + h[2 + 2 * k];
        dm = h[1 + 2 * k] - h[2 + 2 * k];
    }, h[0], m0, jx, jy, pxx, pxy, pyy);
    coef_tail<L, ST, COLL>(P, dv, dv_f, m0, jx, jy, pxx, pxy, pyy, C);
}

// Output of the rest direction, in storage units (the coefficients already carry 1/s).
template <class L, int COLL, class T>
__device__ __forceinline__ T eval_rest(const Coef<T>& C, T h0) {
    if (COLL == COLL_REG) return C.ce[0];
    return h0 + C.om * (C.e0 - h0) + C.ce[0];
}

// Outputs of pair k (+p_k, -p_k), in storage units and relative to the stored state's stream
// offset (16-bit); hp, hm are the pulled populations (BGK only).  The pair tables have p_kx >= 0,
// so m = p_kx indexes the per-|c_x| constants.
template <class L, int COLL, class T>
__device__ __forceinline__ void eval_pair(const Coef<T>& C, int k, T hp, T hm, T& op, T& omn) {
    const int px = L::px(k), py = L::py(k);
    static_assert(L::px(0) >= 0, "pairs are listed with p_x >= 0");
    T a = 0;
    if (px) a += (T)px * C.ax;
    if (py) a += (T)py * C.ay;
    const T a2 = a * a;
    if (COLL == COLL_REG) {
        T E = C.ce[px] + a2 * (C.e1 + a2 * C.e2);
        if (px) E += (T)(px * px) * C.rxx;
        if (px && py) E += (T)(px * py) * C.rxy;
        if (py) E += (T)(py * py) * C.ryy;
        if (px) E += a * ((T)px * C.kf);
        const T O = a * (C.o0 + C.o1 * a2) + C.co[px];
        // Eq. 18: f = f^eq + (1 - 1/tau) f^ne (+ source)
        op = E + O;
        omn = E - O;
    } else {
        const T E = C.e0 + a2 * (C.e1 + a2 * C.e2);
        const T O = a * (C.o0 + C.o1 * a2);
        T Es = C.ce[px];
        if (px) Es += a * ((T)px * C.kf);
        const T Os = C.co[px];
        // Eq. 14 discretized: f - (f - f^eq)/tau + source
        op = hp + C.om * ((E + O) - hp) + (Es + Os);
        omn = hm + C.om * ((E - O) - hm) + (Es - Os);
    }
}

// Two FP32 lanes in one 64-bit register pair, and the packed FP32 operations of sm_100+ (each lane
// rounds to nearest like the scalar operation; one instruction issues both).
struct F2 {
    unsigned long long v;
};
__device__ __forceinline__ F2 f2(float lo, float hi) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_split(F2 a, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
    F2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}

// Outputs of the pairs k and k + 1 of the regularized collision in FP32, two pairs per packed
// operation.  The pair tables list pairs in groups of two that share their arithmetic: (p_x, p_y)
// and (p_x, -p_y), or (m, 0) and (0, m).  Same expressions as eval_pair, evaluated in a different
// order (FP32 rounding differs).
template <class L>
__device__ __forceinline__ void eval_group(const Coef<float>& C, int k, F2 E1, F2 E2, F2 O0, F2 O1, float& op1,
                                           float& om1, float& op2, float& om2) {
    const int px1 = L::px(k), py1 = L::py(k), px2 = L::px(k + 1), py2 = L::py(k + 1);
    float a1, a2, q1, q2, k1, k2, c1, c2;
    if (px1 == px2 && py1 == -py2) {
        // (p_x, +-p_y): a = X +- Y, shared even constant, opposite mixed terms
        const float X = (float)px1 * C.ax, Y = (float)py1 * C.ay;
        a1 = X + Y;
        a2 = X - Y;
        const float B = C.ce[px1] + (float)(px1 * px1) * C.rxx + (float)(py1 * py1) * C.ryy;
        q1 = B + (float)(px1 * py1) * C.rxy;
        q2 = B - (float)(px1 * py1) * C.rxy;
        k1 = k2 = (float)px1 * C.kf;
        c1 = c2 = C.co[px1];
    } else {
        // (m, 0) and (0, m)
        a1 = (float)px1 * C.ax + (float)py1 * C.ay;
        a2 = (float)px2 * C.ax + (float)py2 * C.ay;
        q1 = C.ce[px1] + (float)(px1 * px1) * C.rxx + (float)(py1 * py1) * C.ryy + (float)(px1 * py1) * C.rxy;
        q2 = C.ce[px2] + (float)(px2 * px2) * C.rxx + (float)(py2 * py2) * C.ryy + (float)(px2 * py2) * C.rxy;
        k1 = (float)px1 * C.kf;
        k2 = (float)px2 * C.kf;
        c1 = C.co[px1];
        c2 = C.co[px2];
    }
    const F2 A = f2(a1, a2);
    const F2 A2 = mul2(A, A);
    F2 E = fma2(A2, fma2(A2, E2, E1), f2(q1, q2));
    E = fma2(A, f2(k1, k2), E);
    const F2 O = fma2(A, fma2(O1, A2, O0), f2(c1, c2));
    f2_split(add2(E, O), op1, op2);
    f2_split(sub2(E, O), om1, om2);
}

// Evaluation of one node's outputs from its coefficients; emit(i, v) receives output i in storage
// units (relative to the stream offset when it is on).  The regularized collision in FP32
// evaluates two pairs per packed operation and never reads h; plain BGK reads the pulled h.
template <class L, class ST, int COLL, class Emit>
__device__ __forceinline__ void emit_outputs(const Coef<typename StoreT<ST>::CT>& C,
                                             const typename StoreT<ST>::CT (&h)[L::Q], Emit&& emit) {
    using T = typename StoreT<ST>::CT;
    if constexpr (COLL == COLL_REG) {
        emit(0, C.ce[0]);
    } else {
        emit(0, eval_rest<L, COLL, T>(C, h[0]));
    }
    if constexpr (COLL == COLL_REG && sizeof(T) == 4 && L::NP % 2 == 0) {
        const F2 E1 = f2(C.e1, C.e1), E2 = f2(C.e2, C.e2), O0 = f2(C.o0, C.o0), O1 = f2(C.o1, C.o1);
#pragma unroll
        for (int k = 0; k < L::NP; k += 2) {
            float op1, om1, op2, om2;
            eval_group<L>(C, k, E1, E2, O0, O1, op1, om1, op2, om2);
            emit(1 + 2 * k, op1);
            emit(2 + 2 * k, om1);
            emit(3 + 2 * k, op2);
            emit(4 + 2 * k, om2);
        }
    } else {
#pragma unroll
        for (int k = 0; k < L::NP; ++k) {
            T op, omn;
            if constexpr (COLL == COLL_REG)
                eval_pair<L, COLL, T>(C, k, (T)0, (T)0, op, omn);
            else
                eval_pair<L, COLL, T>(C, k, h[1 + 2 * k], h[2 + 2 * k], op, omn);
            emit(1 + 2 * k, op);
            emit(2 + 2 * k, omn);
        }
    }
}

// prepare + evaluation of one node (see emit_outputs).
template <class L, class ST, int COLL, int WALL = 0, bool COH = false, class Emit>
__device__ __forceinline__ void collide_emit(const InstDev& P, const void* src_v, int x, int y, int cls, double dv,
                                             float dv_f, typename StoreT<ST>::CT (&h)[L::Q], double& Fx, double& Fy,
                                             Emit&& emit) {
    Coef<typename StoreT<ST>::CT> C;
    prepare<L, ST, COLL, WALL, OWN_OPP, COH>(P, src_v, x, y, cls, dv, dv_f, h, Fx, Fy, C);
    emit_outputs<L, ST, COLL>(C, h, emit);
}

// prepare + evaluation + store of one node.
template <class L, class ST, int COLL, int WALL = 0, bool COH = false>
__device__ __forceinline__ void collide_store(const InstDev& P, const void* src_v, void* dst_v, int x, int y, int cls,
                                              double dv, float dv_f, typename StoreT<ST>::CT (&h)[L::Q], double& Fx,
                                              double& Fy) {
    using S = StoreT<ST>;
    using T = typename S::CT;
    // 32-bit plane stride (Q * plane < 2^32, checked at creation): each address is the node's
    // pointer plus stride * i, one widening multiply-add
    ST* __restrict__ dst = static_cast<ST*>(dst_v) + (y * P.pitch + x);
    const unsigned plane = (unsigned)P.plane;
    collide_emit<L, ST, COLL, WALL, COH>(P, src_v, x, y, cls, dv, dv_f, h, Fx, Fy,
                                         [&](int i, T v) { S::stg(dst + (unsigned long long)plane * (unsigned)i, v); });
}

// Advection + wall + collision of the fluid node (x, y), sources from global memory.  WALL selects
// bounce-back (0) or diffuse scattering (1) at compile time: the diffuse fix-up costs registers
// that the bulk of the nodes must not pay for.
template <class L, class ST, int COLL, int WALL = 0>
__device__ __forceinline__ void node_update(const InstDev& P, const void* src, void* dst, int x, int y, int cls,
                                            double dv, float dv_f, double& Fx, double& Fy) {
    typename StoreT<ST>::CT h[L::Q];
    gather_global<L, ST>(P, static_cast<const ST*>(src), x, y, h);
    collide_store<L, ST, COLL, WALL>(P, src, dst, x, y, cls, dv, dv_f, h, Fx, Fy);
}

// Force partial of a tile (fixed-order reduction); the last tile with body links to finish sums
// the slots in a fixed order, adds the constant part and writes the force of the step.  Returns
// true (block-uniform) in the block that wrote the force.
template <int NF>
__device__ __forceinline__ bool tile_epilogue_n(const InstDev& P, int slot, double2* force_out, double (&F)[2 * NF]) {
    if (slot < 0) return false;  // block-uniform: no body link in this tile
    __shared__ double2 red[32 * NF];
    __shared__ int last;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nwarps = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
#pragma unroll
        for (int c = 0; c < 2 * NF; ++c) F[c] += __shfl_down_sync(0xffffffffu, F[c], o);
    }
    if ((tid & 31) == 0) {
#pragma unroll
        for (int f = 0; f < NF; ++f) red[(tid >> 5) * NF + f] = make_double2(F[2 * f], F[2 * f + 1]);
    }
    __syncthreads();
    if (tid < 32) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            double2 v = tid < nwarps ? red[tid * NF + f] : make_double2(0.0, 0.0);
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                v.x += __shfl_down_sync(0xffffffffu, v.x, o);
                v.y += __shfl_down_sync(0xffffffffu, v.y, o);
            }
            if (tid == 0) P.partials[slot * NF + f] = v;
        }
        if (tid == 0) {
            __threadfence();
            const unsigned t = atomicAdd(P.ticket, 1u);
            last = (t == (unsigned)(P.nslots - 1));
        }
    }
    __syncthreads();
    if (last && tid < 32) {
        __threadfence();
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            double sx = 0.0, sy = 0.0;
            for (int k = tid; k < P.nslots; k += 32) {
                const double2 v = __ldcg(P.partials + k * NF + f);
                sx += v.x;
                sy += v.y;
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                sx += __shfl_down_sync(0xffffffffu, sx, o);
                sy += __shfl_down_sync(0xffffffffu, sy, o);
            }
            if (tid == 0) {
                const double2 Fs = make_double2(sx + P.fconst.x, sy + P.fconst.y);
                if (!isfinite(Fs.x) || !isfinite(Fs.y)) atomicOr(P.err, 1);
                force_out[f] = Fs;
            }
        }
        if (tid == 0) *P.ticket = 0u;
    }
    return last != 0;
}

__device__ __forceinline__ bool tile_epilogue(const InstDev& P, int slot, double2* force_out, double Fx, double Fy) {
    double F[2] = {Fx, Fy};
    return tile_epilogue_n<1>(P, slot, force_out, F);
}

// Node (x, y) inside the grid, of class cls (already loaded).  With 4- and 8-byte storage its pulls
// are issued whatever the class (the pulls of any node inside the grid are in bounds, so they need
// not wait for the class test), then a fluid node collides and stores; solid nodes load for
// nothing, a small fraction of a grid.  The 16-bit kernels run at a register budget where that
// spills, so they test the class first.
template <class L, class ST, int COLL, int WALL = 0>
__device__ __forceinline__ void node_update_cls(const InstDev& P, const void* src, void* dst, int x, int y, int cls,
                                                double dv, float dv_f, double& Fx, double& Fy) {
    if constexpr (sizeof(ST) == 2) {
        if (cls != NODE_SOLID) node_update<L, ST, COLL, WALL>(P, src, dst, x, y, cls, dv, dv_f, Fx, Fy);
    } else {
        typename StoreT<ST>::CT h[L::Q];
        gather_global<L, ST>(P, static_cast<const ST*>(src), x, y, h);
        if (cls != NODE_SOLID) collide_store<L, ST, COLL, WALL>(P, src, dst, x, y, cls, dv, dv_f, h, Fx, Fy);
    }
}

// One tile of one instance: blockDim.x * blockDim.y nodes, one thread per node.  PDL: the kernel
// was launched with programmatic stream serialization; the node's class (geometry, written by the
// host only) is read before the wait for the previous step's grid, the populations after it.
template <class L, class ST, int COLL, int WALL = 0, bool PDL = false>
__device__ __forceinline__ void process_tile(const InstDev& P, int tile, const void* src, void* dst, double dv,
                                             float dv_f, double2* force_out) {
    const int tx = tile % P.ntx, ty = tile / P.ntx;
    const int x = tx * blockDim.x + threadIdx.x;
    const int y = ty * blockDim.y + threadIdx.y;
    // 16-bit kernels read their tile's slot early, so that the epilogue need not wait for it; the
    // 4- and 8-byte kernels have no register left for it (it spilled) and read it at the end
    int slot = sizeof(ST) == 2 ? P.tile_slot[tile] : 0;
    const bool inside = x < P.nx && y < P.ny;
    const int cls = inside ? (int)P.cls[y * P.pitch + x] : (int)NODE_SOLID;
    if (PDL) pdl_wait_then_release();
    double Fx = 0.0, Fy = 0.0;
    if (inside) node_update_cls<L, ST, COLL, WALL>(P, src, dst, x, y, cls, dv, dv_f, Fx, Fy);
    if (sizeof(ST) != 2) slot = P.tile_slot[tile];
    tile_epilogue(P, slot, force_out, Fx, Fy);
}

// Single-instance step: one block per tile.
template <class L, class ST, int COLL, int WALL = 0>
__global__ void __launch_bounds__(512) step_kernel(const __grid_constant__ InstDev P) {
    process_tile<L, ST, COLL, WALL, true>(P, blockIdx.x, P.src, P.dst, P.dv, P.dv_f, P.force_out);
}

using StepLaunchFn = cudaError_t (*)(const InstDev& P, dim3 block, cudaStream_t stream);

template <class L, class ST, int COLL, int WALL = 0>
cudaError_t launch_step(const InstDev& P, dim3 block, cudaStream_t stream) {
    return launch_pdl(step_kernel<L, ST, COLL, WALL>, dim3(P.ntiles), block, 0, stream, P);
}

// The plain step on 32 x 4 tiles with an occupancy floor: at least MINB blocks of 128 threads per
// SM, so the compiler keeps the kernel within 65536 / (128 MINB) registers per thread.  The plain
// kernel waits on its global loads; more resident warps hide more of that latency.
template <class L, class ST, int COLL, int MINB>
__global__ void __launch_bounds__(128, MINB) step_kernel_occ(const __grid_constant__ InstDev P) {
    process_tile<L, ST, COLL, 0, true>(P, blockIdx.x, P.src, P.dst, P.dv, P.dv_f, P.force_out);
}

template <class L, class ST, int COLL, int MINB>
cudaError_t launch_step_occ(const InstDev& P, dim3 block, cudaStream_t stream) {
    return launch_pdl(step_kernel_occ<L, ST, COLL, MINB>, dim3(P.ntiles), block, 0, stream, P);
}

// The same on tiles of 32 x (4 NR) nodes: each thread computes NR nodes of its column, 4 rows apart,
// one at a time, so that the block's fixed costs (tile indices, launch constants, the force
// epilogue) are spread over NR nodes.
template <class L, class ST, int COLL, int MINB, int NR>
__global__ void __launch_bounds__(128, MINB) step_kernel_occn(const __grid_constant__ InstDev P) {
    pdl_wait_then_release();
    const int t = blockIdx.x;
    const int x = (t % P.ntx) * 32 + threadIdx.x;
    const int y0 = (t / P.ntx) * (4 * NR) + threadIdx.y;
    const int slot = P.tile_slot[t];
    double Fx = 0.0, Fy = 0.0;
#pragma unroll 1
    for (int r = 0; r < NR; ++r) {
        const int y = y0 + 4 * r;
        if (x < P.nx && y < P.ny)
            node_update_cls<L, ST, COLL, 0>(P, P.src, P.dst, x, y, (int)P.cls[y * P.pitch + x], P.dv, P.dv_f, Fx, Fy);
    }
    tile_epilogue(P, slot, P.force_out, Fx, Fy);
}

template <class L, class ST, int COLL, int MINB, int NR>
cudaError_t launch_step_occn(const InstDev& P, dim3, cudaStream_t stream) {
    return launch_pdl(step_kernel_occn<L, ST, COLL, MINB, NR>, dim3(P.ntiles), dim3(32, 4), 0, stream, P);
}

// Launchers for (lattice Q, storage, collision); nullptr if the combination is not built.
StepLaunchFn find_step_launcher(int Q, int storage, int coll, int wall = 0);
// Plain step with an occupancy floor: variant 1 = 6 blocks of 128 per SM, 2 = 7; 3, 4 = 7 blocks with
// 2 or 4 nodes per thread (nullptr if not built).
StepLaunchFn find_occ_launcher(int Q, int storage, int coll, int variant);

}  // namespace lbm
