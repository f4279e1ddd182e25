// Per-node arithmetic of the explicit schemes of arXiv:1904.04048, Section 6.
//
// Every kernel of the library (one-node-per-thread, TMA tiles, temporal
// blocking, batched) evaluates a node through the functions in this file, with
// the operations pinned to round-to-nearest intrinsics so the compiler cannot
// contract or reorder them differently from one kernel to the next.  The
// results of different tilings are therefore bitwise identical.
//
// Stencil sums (Eq. notations2, read with i - q1 in the third term):
//   delta(1,0) = ((e + w) + (n + s)) - 4c
//   delta(1,1) = ((ne + sw) + (nw + se)) - 4c
//   delta(2,0) = ((ee + ww) + (nn + ss)) - 4c
// The pairing of opposite neighbours makes each sum invariant under the eight
// symmetries of the square grid bit for bit (every rotation or reflection
// only swaps operands of a commutative addition).
#pragma once
#include <type_traits>
#include <cstdint>

namespace w2d {

// ----------------------------------------------------------------------------
// Double-float ("FP32x2") value: an unevaluated sum hi + lo with
// |lo| <= ulp(hi)/2.  Error-free transforms: TwoSum (Knuth), Fast2Sum
// (Dekker 1971), TwoProd with a fused multiply-add.  Addition is Dekker's
// double-length sum (one TwoSum of the high parts, the low parts added in,
// one Fast2Sum): its error is a few units of 2^-48 of |x| + |y| rather than
// of |x + y|.  Every sum of the schemes is added, directly or after a
// coefficient product, to 2u^k - u^{k-1}, so what matters is the error
// relative to the field, which this bound gives; it takes 11 FP32 operations
// where the TwoSum-of-both-parts form takes 20.
// ----------------------------------------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
// Double-float addition (Dekker's double-length sum).
__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    float e = __fadd_rn(__fadd_rn(s.lo, x.lo), y.lo);
    return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
// Product of two double-float numbers (the low-times-low term is dropped).
__device__ __forceinline__ df df_mul(df a, df x) {
    float p = __fmul_rn(a.hi, x.hi);
    float e = __fmaf_rn(a.hi, x.hi, -p);
    e = __fmaf_rn(a.hi, x.lo, e);
    e = __fmaf_rn(a.lo, x.hi, e);
    return fast_two_sum(p, e);
}
// Scaling by a power of two is exact.
__device__ __forceinline__ df df_scale(df x, float s) { return {__fmul_rn(x.hi, s), __fmul_rn(x.lo, s)}; }

// ----------------------------------------------------------------------------
// Uniform operation set over float, double and df.
// ----------------------------------------------------------------------------
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ df vadd(df a, df b) { return df_add(a, b); }

__device__ __forceinline__ float vscale(float a, float s) { return __fmul_rn(a, s); }
__device__ __forceinline__ double vscale(double a, float s) { return __dmul_rn(a, (double)s); }
__device__ __forceinline__ df vscale(df a, float s) { return df_scale(a, s); }

// a * d + acc
__device__ __forceinline__ float vfma(float a, float d, float acc) { return __fmaf_rn(a, d, acc); }
__device__ __forceinline__ double vfma(double a, double d, double acc) { return __fma_rn(a, d, acc); }
__device__ __forceinline__ df vfma(df a, df d, df acc) { return df_add(df_mul(a, d), acc); }

__device__ __forceinline__ float vmul(float a, float d) { return __fmul_rn(a, d); }
__device__ __forceinline__ double vmul(double a, double d) { return __dmul_rn(a, d); }
__device__ __forceinline__ df vmul(df a, df d) { return df_mul(a, d); }

__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double vsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ df vsub(df a, df b) { return df_add(a, df_neg(b)); }

// x + s a for a power-of-two s (s a exact): for float and double one fused
// multiply-add, which rounds once exactly as the sum x + (s a) does; for
// double-float the sum itself, in that operand order.
__device__ __forceinline__ float vadd_scaled(float x, float a, float s) { return __fmaf_rn(a, s, x); }
__device__ __forceinline__ double vadd_scaled(double x, double a, float s) { return __fma_rn(a, (double)s, x); }
__device__ __forceinline__ df vadd_scaled(df x, df a, float s) { return df_add(x, df_scale(a, s)); }

// 2 c - p: one rounding (2 c is exact); the double-float form subtracts.
__device__ __forceinline__ float vtwo_minus(float c, float p) { return __fmaf_rn(c, 2.0f, -p); }
__device__ __forceinline__ double vtwo_minus(double c, double p) { return __fma_rn(c, 2.0, -p); }
__device__ __forceinline__ df vtwo_minus(df c, df p) { return df_add(df_scale(c, 2.0f), df_neg(p)); }

template <typename V>
struct Coef3 {
    V a10, a11, a20;
};

// Values of one level around a node.  n/s are rows j+1 / j-1, e/w columns
// i+1 / i-1; the second ring (ee, ww, nn, ss) is used by the 13-point scheme.
template <typename V>
struct Nbr {
    V c, e, w, n, s, ne, nw, se, sw, ee, ww, nn, ss;
};

// Each class sum adds its -4 u_ij term last (vadd_scaled: one rounding, the
// same as adding the exact product -4 u_ij).  Double-float forms -4 u_ij once
// and adds it to each class sum (the same operations as vadd_scaled; measured
// on GB300, the 13-point FP32x2 level takes 164 us at 4096^2 this way and 178
// with the product written into every class sum).
template <int S, typename V>
__device__ __forceinline__ V lambda_sum(const Nbr<V>& u, const Coef3<V>& a) {
    if constexpr (std::is_same_v<V, df>) {
        const df m4c = df_scale(u.c, -4.0f);
        df d10 = df_add(vadd(vadd(u.e, u.w), vadd(u.n, u.s)), m4c);
        df L = vmul(a.a10, d10);
        if constexpr (S >= 9) {
            df d11 = df_add(vadd(vadd(u.ne, u.sw), vadd(u.nw, u.se)), m4c);
            L = vfma(a.a11, d11, L);
        }
        if constexpr (S == 13) {
            df d20 = df_add(vadd(vadd(u.ee, u.ww), vadd(u.nn, u.ss)), m4c);
            L = vfma(a.a20, d20, L);
        }
        return L;
    } else {
        V d10 = vadd_scaled(vadd(vadd(u.e, u.w), vadd(u.n, u.s)), u.c, -4.0f);
        V L = vmul(a.a10, d10);
        if constexpr (S >= 9) {
            V d11 = vadd_scaled(vadd(vadd(u.ne, u.sw), vadd(u.nw, u.se)), u.c, -4.0f);
            L = vfma(a.a11, d11, L);
        }
        if constexpr (S == 13) {
            V d20 = vadd_scaled(vadd(vadd(u.ee, u.ww), vadd(u.nn, u.ss)), u.c, -4.0f);
            L = vfma(a.a20, d20, L);
        }
        return L;
    }
}

// Two-step (Eq. A2): u^{k+1} = (2 u^k - u^{k-1}) + Lambda_a(u^k), with
// Lambda_a accumulated on its own (its magnitude is far below that of u for
// smooth fields) and added to 2u^k - u^{k-1} by a single rounding.  Adding
// each coefficient's term to the base in turn (a chain of FMAs onto
// 2u^k - u^{k-1}) was measured to let FP32 rounding drift up to 48 times
// faster over 10^4 steps for long waves, so this order is kept.
template <int S, typename V>
__device__ __forceinline__ V two_step_update(const Nbr<V>& u, V prev, const Coef3<V>& a) {
    V L = lambda_sum<S>(u, a);
    V base = vtwo_minus(u.c, prev);
    return vadd(base, L);
}

// First step (Eq. A1), always in FP64:
// u^1 = (u^0 + tau v^0) + (Lambda_{a/2}(u^0) + tau Lambda_b(v^0)).
template <int S>
__device__ __forceinline__ double first_step_update(const Nbr<double>& u, const Nbr<double>& v,
                                                    const Coef3<double>& ahalf,
                                                    const Coef3<double>& b, double tau) {
    double Lu = lambda_sum<S>(u, ahalf);
    double Lv = lambda_sum<S>(v, b);
    return __dadd_rn(__fma_rn(tau, v.c, u.c), __fma_rn(tau, Lv, Lu));
}

// ----------------------------------------------------------------------------
// Two neighbouring nodes at once with the packed FP32 instructions of sm_100+
// (add/mul/fma .rn.f32x2).  Every lane performs exactly the rounding steps of
// two_step_update on float, in the same order, so the results are bitwise
// those of the scalar path.
// ----------------------------------------------------------------------------
typedef unsigned long long f2x;

__device__ __forceinline__ f2x pk2(float lo, float hi) {
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(f2x v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
    f2x d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
    f2x d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
    f2x d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Rows hold x-2 .. x+5 of one 4-node vector (a[k] = column x + k - 2); the
// pair starts at node e (0 or 2).  up/dn are rows j+1 / j-1, up2/dn2 rows
// j+2 / j-2 (13-point only).  Coefficients arrive as duplicated pairs.
// Packed pair for the 9- and 13-point schemes.  The final addition consumes
// the result of an FMA (a11 or a20 term), which no compiler can merge into the
// product before it, so every lane rounds exactly as two_step_update does.
// (For the 5-point scheme the last product would feed the addition directly,
// and a packed multiply followed by a packed add may be fused: that scheme
// uses the scalar path.)
// Operand pairs that start at an even column (the centre, the north/south and
// second-ring neighbours) are register pairs of the row buffers and enter the
// packed instructions as they are; the east/west and diagonal neighbours of
// the two nodes start at an odd column, so their pair sums are formed by two
// scalar additions (the same roundings) whose results make a register pair,
// instead of moving misaligned operands into pairs first.
template <int S>
__device__ __forceinline__ void two_step_update_pair(const float* c, const float* up, const float* dn,
                                                     const float* up2, const float* dn2, int e, float p0,
                                                     float p1, f2x a10, f2x a11, f2x a20, float& o0,
                                                     float& o1) {
    static_assert(S == 9 || S == 13, "packed pair path is for the 9- and 13-point schemes");
    const f2x cc = pk2(c[e + 2], c[e + 3]);
    const f2x m4 = pk2(-4.0f, -4.0f);
    // Each class sum ends with the -4 u_ij term as one FMA, cc * (-4) + sum:
    // -4 u_ij is exact, so this rounds once, exactly as the scalar path's
    // sum + (-4 u_ij) does, and saves the separate product.
    // delta(1,0): (east + west) + (north + south)
    const f2x ew = pk2(__fadd_rn(c[e + 3], c[e + 1]), __fadd_rn(c[e + 4], c[e + 2]));
    const f2x ns = add2(pk2(up[e + 2], up[e + 3]), pk2(dn[e + 2], dn[e + 3]));
    const f2x d10 = fma2(cc, m4, add2(ew, ns));
    f2x L = mul2(a10, d10);
    // delta(1,1): (ne + sw) + (nw + se)
    const f2x nesw = pk2(__fadd_rn(up[e + 3], dn[e + 1]), __fadd_rn(up[e + 4], dn[e + 2]));
    const f2x nwse = pk2(__fadd_rn(up[e + 1], dn[e + 3]), __fadd_rn(up[e + 2], dn[e + 4]));
    const f2x d11 = fma2(cc, m4, add2(nesw, nwse));
    L = fma2(a11, d11, L);
    if constexpr (S == 13) {
        // delta(2,0): (ee + ww) + (nn + ss), all pairs even-aligned
        const f2x d20 = fma2(cc, m4, add2(add2(pk2(c[e + 4], c[e + 5]), pk2(c[e], c[e + 1])),
                                          add2(pk2(up2[e + 2], up2[e + 3]), pk2(dn2[e + 2], dn2[e + 3]))));
        L = fma2(a20, d20, L);
    }
    const f2x base = fma2(pk2(p0, p1), pk2(-1.0f, -1.0f), mul2(cc, pk2(2.0f, 2.0f)));
    upk2(add2(base, L), o0, o1);
}

}  // namespace w2d
