// lattice.cuh -- velocity sets of the GPU path, as compile-time constants.
//
// D2Q37: Appendix A, Table "D2Q37" (8 shells, weights to 15-18 digits, lattice speed
// c = 1.19697977039307 sqrt(theta)); lattice units with c = 1, so theta = 1/1.19697977039307^2.
// D2Q9: the textbook nine-velocity lattice (theta = 1/3); the paper does not use it.
//
// Direction order used everywhere on the GPU side: 0 is the rest velocity, then pairs
// (1 + 2k, 2 + 2k) = (+p_k, -p_k) for k = 0 .. NP-1.  The +/- pairing lets the collision evaluate
// the even and odd parts of each polynomial once per pair.
#pragma once

namespace lbm {

struct D2Q9 {
    static constexpr int Q = 9;
    static constexpr int NP = 4;   // velocity pairs
    static constexpr int R = 1;    // largest |c_ia|
    __host__ __device__ static constexpr double theta() { return 1.0 / 3.0; }
    __host__ __device__ static constexpr double w0() { return 4.0 / 9.0; }
    __host__ __device__ static constexpr int px(int k) { return k == 0 ? 1 : k == 1 ? 0 : k == 2 ? 1 : 1; }
    __host__ __device__ static constexpr int py(int k) { return k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 1 : -1; }
    __host__ __device__ static constexpr double wp(int k) { return k < 2 ? 1.0 / 9.0 : 1.0 / 36.0; }
};

struct D2Q37 {
    static constexpr int Q = 37;
    static constexpr int NP = 18;
    static constexpr int R = 3;
    __host__ __device__ static constexpr double theta() {
        return 1.0 / (1.19697977039307 * 1.19697977039307);
    }
    __host__ __device__ static constexpr double w0() { return 0.233150669132352000; }
    // shells (1,0) (1,1) (2,0) (2,2) (3,0) with two pairs each, then (1,2) and (1,3) with four
    __host__ __device__ static constexpr int px(int k) {
        return k == 0 ? 1 : k == 1 ? 0 : k == 2 ? 1 : k == 3 ? 1 : k == 4 ? 2 : k == 5 ? 0 : k == 6 ? 2
             : k == 7 ? 2 : k == 8 ? 3 : k == 9 ? 0 : k == 10 ? 1 : k == 11 ? 1 : k == 12 ? 2 : k == 13 ? 2
             : k == 14 ? 1 : k == 15 ? 1 : k == 16 ? 3 : 3;
    }
    __host__ __device__ static constexpr int py(int k) {
        return k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 1 : k == 3 ? -1 : k == 4 ? 0 : k == 5 ? 2 : k == 6 ? 2
             : k == 7 ? -2 : k == 8 ? 0 : k == 9 ? 3 : k == 10 ? 2 : k == 11 ? -2 : k == 12 ? 1 : k == 13 ? -1
             : k == 14 ? 3 : k == 15 ? -3 : k == 16 ? 1 : -1;
    }
    __host__ __device__ static constexpr double wp(int k) {
        return k < 2 ? 0.107306091542219000
             : k < 4 ? 0.057667859888794800
             : k < 6 ? 0.014208216158450700
             : k < 8 ? 0.001011937592673570
             : k < 10 ? 0.000245301027757717
             : k < 14 ? 0.005353049000513770
             : 0.000283414252994198;
    }
};

// Velocity and weight of direction i in the GPU order.
template <class L>
__host__ __device__ constexpr int cx_of(int i) { return i == 0 ? 0 : ((i - 1) & 1 ? -L::px((i - 1) >> 1) : L::px((i - 1) >> 1)); }
template <class L>
__host__ __device__ constexpr int cy_of(int i) { return i == 0 ? 0 : ((i - 1) & 1 ? -L::py((i - 1) >> 1) : L::py((i - 1) >> 1)); }
template <class L>
__host__ __device__ constexpr double w_of(int i) { return i == 0 ? L::w0() : L::wp((i - 1) >> 1); }
template <class L>
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : ((i - 1) & 1 ? i - 1 : i + 1); }

}  // namespace lbm
