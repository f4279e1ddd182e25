// Per-node arithmetic of the derived schemes: the construction of Sections
// 4-5 of arXiv:1904.04048 applied to larger monomial segments M*_{<=m}.
//
// Where the derived weights are symmetric under the eight symmetries of the
// square, a scheme is a sum over classes of nodes: class (q1, q2), with
// q1 > 0 and 0 <= q2 <= q1, holds the nodes (+-q1, +-q2) and (+-q2, +-q1)
// (four of them when q2 == 0 or q2 == q1, else eight).  Growing segments bring
// the classes in a fixed order, the class chain
//     (1,0) (1,1) (2,0) (2,1) (3,0) (2,2) (3,1) (4,0)
// (m = 6: 5 points, 11: 9, 15: 13, 24: 21, 28: 25, 37: 29, 41: 37, 45: 41),
// so a scheme is a prefix of NC classes with one coefficient each:
//   Lambda_a(u) = sum_c a_c delta_c(u),  delta_c = (sum of u over class c) - n_c u_ij.
// The two-step (Eq. A2) is u^{k+1} = (2u^k - u^{k-1}) + Lambda_a(u^k), the
// first step (Eq. A1) u^1 = (u^0 + tau v^0) + (Lambda_{a/2}(u^0) + tau Lambda_b(v^0)).
//
// Rounding: every class sum pairs opposite nodes, ((q + -q) + (r + -r)) for
// the two rotations of a four-node orbit and the sum of the two orbits'
// sums for an eight-node class, so every symmetry of the square only swaps
// operands of commutative additions and the result is equivariant bit for
// bit.  For NC <= 3 the operations are exactly those of the Section 6
// schemes in stencil_ops.cuh, in the same order.
//
// Difference sums (DIFF = true): each node enters as its difference to the
// centre, delta_c = ((u_q - u_ij) + (u_-q - u_ij)) + ((u_r - u_ij) + (u_-r - u_ij)).
// For a smooth field, away from its zeros, a neighbour and the centre are
// within a factor two of each other, so each difference is exact (Sterbenz's
// lemma) and the rounding error of delta is relative to delta itself, not to
// u: for long
// waves (delta ~ (omega tau)^2 u) this keeps the bits the plain sum loses to
// cancellation.  Same pairing, so the same bitwise symmetry.
#pragma once
#include "stencil_ops.cuh"

namespace w2d {

constexpr int kMaxClasses = 8;

__host__ __device__ constexpr int chain_q1(int c) {
    return c == 0 ? 1 : c == 1 ? 1 : c == 2 ? 2 : c == 3 ? 2 : c == 4 ? 3 : c == 5 ? 2 : c == 6 ? 3 : 4;
}
__host__ __device__ constexpr int chain_q2(int c) {
    return c == 0 ? 0 : c == 1 ? 1 : c == 2 ? 0 : c == 3 ? 1 : c == 4 ? 0 : c == 5 ? 2 : c == 6 ? 1 : 0;
}
__host__ __device__ constexpr int chain_nodes(int c) {
    return (chain_q2(c) == 0 || chain_q2(c) == chain_q1(c)) ? 4 : 8;
}
// Stencil radius of the first nc classes.
__host__ __device__ constexpr int chain_radius(int nc) {
    int r = 0;
    for (int c = 0; c < nc; ++c) r = chain_q1(c) > r ? chain_q1(c) : r;
    return r;
}
// Number of stencil nodes (centre included) of the first nc classes.
__host__ __device__ constexpr int chain_points(int nc) {
    int n = 1;
    for (int c = 0; c < nc; ++c) n += chain_nodes(c);
    return n;
}

template <typename V, int NC>
struct CoefN {
    V a[NC];
};

// delta_c of class C at a node; u(dx, dy) returns the level at offset
// (dx, dy) (dx along x1 = columns, dy along x2 = rows).
template <int C, bool DIFF, typename V, typename F>
__device__ __forceinline__ V class_delta(const F& u, V c) {
    constexpr int q1 = chain_q1(C), q2 = chain_q2(C);
    if constexpr (DIFF) {
        const auto d = [&](int x, int y) { return vsub(u(x, y), c); };
        V s = vadd(vadd(d(q1, q2), d(-q1, -q2)), vadd(d(-q2, q1), d(q2, -q1)));
        if constexpr (chain_nodes(C) == 8) {
            const V t = vadd(vadd(d(q2, q1), d(-q2, -q1)), vadd(d(-q1, q2), d(q1, -q2)));
            s = vadd(s, t);
        }
        return s;
    } else {
        V s = vadd(vadd(u(q1, q2), u(-q1, -q2)), vadd(u(-q2, q1), u(q2, -q1)));
        if constexpr (chain_nodes(C) == 8) {
            const V t = vadd(vadd(u(q2, q1), u(-q2, -q1)), vadd(u(-q1, q2), u(q1, -q2)));
            s = vadd(s, t);
        }
        return vadd_scaled(s, c, -(float)chain_nodes(C));
    }
}

template <int NC, bool DIFF = false, typename V, typename F>
__device__ __forceinline__ V lambda_chain(const F& u, V c, const CoefN<V, NC>& a) {
    static_assert(NC >= 1 && NC <= kMaxClasses, "class count");
    V L = vmul(a.a[0], class_delta<0, DIFF>(u, c));
    if constexpr (NC > 1) L = vfma(a.a[1], class_delta<1, DIFF>(u, c), L);
    if constexpr (NC > 2) L = vfma(a.a[2], class_delta<2, DIFF>(u, c), L);
    if constexpr (NC > 3) L = vfma(a.a[3], class_delta<3, DIFF>(u, c), L);
    if constexpr (NC > 4) L = vfma(a.a[4], class_delta<4, DIFF>(u, c), L);
    if constexpr (NC > 5) L = vfma(a.a[5], class_delta<5, DIFF>(u, c), L);
    if constexpr (NC > 6) L = vfma(a.a[6], class_delta<6, DIFF>(u, c), L);
    if constexpr (NC > 7) L = vfma(a.a[7], class_delta<7, DIFF>(u, c), L);
    return L;
}

// Two-step (Eq. A2): (2u^k - u^{k-1}) + Lambda_a(u^k), Lambda accumulated on
// its own and added once (the order of two_step_update).
template <int NC, bool DIFF = false, typename V, typename F>
__device__ __forceinline__ V two_step_chain(const F& u, V c, V prev, const CoefN<V, NC>& a) {
    const V L = lambda_chain<NC, DIFF>(u, c, a);
    const V base = vtwo_minus(c, prev);
    return vadd(base, L);
}

// Difference form of the two-step (the same recursion, Eq. A2, on the pair
// u^k, d^k = u^k - u^{k-1}):  d^{k+1} = d^k + Lambda_a(u^k),
// u^{k+1} = u^k + d^{k+1}.  The small increment Lambda is added to the small
// d, and the rounding of u^{k+1} enters u once instead of being integrated
// twice by the recursion.
template <int NC, bool DIFF, typename V, typename F>
__device__ __forceinline__ void two_step_chain_dform(const F& u, V c, V d, const CoefN<V, NC>& a, V& u_next,
                                                     V& d_next) {
    const V L = lambda_chain<NC, DIFF>(u, c, a);
    d_next = vadd(d, L);
    u_next = vadd(c, d_next);
}

// First step (Eq. A1), FP64.
template <int NC, typename FU, typename FV>
__device__ __forceinline__ double first_step_chain(const FU& u, const FV& v, double uc, double vc,
                                                   const CoefN<double, NC>& ahalf,
                                                   const CoefN<double, NC>& b, double tau) {
    const double Lu = lambda_chain<NC>(u, uc, ahalf);
    const double Lv = lambda_chain<NC>(v, vc, b);
    return __dadd_rn(__fma_rn(tau, vc, uc), __fma_rn(tau, Lv, Lu));
}

}  // namespace w2d
