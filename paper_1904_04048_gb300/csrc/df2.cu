// Two-step (Eq. A2) on double-float storage ("FP32x2", hi + lo planes), two
// neighbouring nodes per thread in packed f32x2 arithmetic.
//
// The double-float level is bound by FP32 arithmetic (about 200 operations
// per 13-point node-update: the error-free sums of stencil_ops.cuh), and the
// one-node kernel spends as many issue slots again on loads, addresses and
// moves: measured on GB300 at 4096^2, issue 78 % active with 3.8 eligible
// warps per scheduler, 167 us per level.  Here a thread updates nodes i and
// i + 1 of up to four consecutive rows: every double-float operation whose operands are register
// pairs (the centre, the north/south and second-ring neighbours, the
// coefficient products, 2u^k - u^{k-1}, the final sum) runs as packed
// add/sub/mul/fma .rn.f32x2, one instruction for both nodes, and the rows
// arrive as 8-byte loads.  Sums whose operands straddle a register pair (east
// + west and the diagonals) run as scalar double-float sums per node, whose
// results then form a pair.
//
// Bitwise equality with the one-node kernel: each lane performs the
// operations of lambda_sum / two_step_update on df (stencil_ops.cuh) in the
// same order with the same roundings.  Subtractions of a negated operand use
// the identities a + (-b) = a - b and -(x) rounded = -(x rounded), both exact
// in IEEE arithmetic, so a packed subtraction replaces an addition of a
// negated value without changing a bit.  Explicit .rn operations are not
// contracted into fused operations.
#include "kernels.cuh"
#include "wave2d_impl.cuh"

namespace w2d {

namespace {

__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
    f2x d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

struct df2 {
    f2x hi, lo;  // lane 0: node i, lane 1: node i + 1
};

__device__ __forceinline__ f2x dup2(float v) { return pk2(v, v); }

// TwoSum, Fast2Sum and Dekker's double-length sum lane by lane (df_add).
__device__ __forceinline__ df2 df2_add(const df2& x, const df2& y) {
    const f2x s = add2(x.hi, y.hi);
    const f2x bb = sub2(s, x.hi);
    const f2x t = add2(sub2(x.hi, sub2(s, bb)), sub2(y.hi, bb));
    const f2x e = add2(add2(t, x.lo), y.lo);
    const f2x h = add2(s, e);
    return {h, sub2(e, sub2(h, s))};
}
// df_add(x, df_neg(y)): x.hi + (-y.hi) = x.hi - y.hi; (-y.hi) - bb =
// -(y.hi + bb), added as a subtraction; the low parts likewise.
__device__ __forceinline__ df2 df2_sub(const df2& x, const df2& y) {
    const f2x s = sub2(x.hi, y.hi);
    const f2x bb = sub2(s, x.hi);
    const f2x t = sub2(sub2(x.hi, sub2(s, bb)), add2(y.hi, bb));
    const f2x e = sub2(add2(t, x.lo), y.lo);
    const f2x h = add2(s, e);
    return {h, sub2(e, sub2(h, s))};
}
// df_mul(a, x) with a a coefficient (the same for both lanes).  The product
// p = a.hi x.hi is carried negated, pn = (-a.hi) x.hi = -p exactly, so that
// fma(a.hi, x.hi, -p) takes pn as its addend; the closing Fast2Sum of p and
// the error e is then s = e - pn (= p + e), err = e - (s + pn) (= e - (s - p)).
__device__ __forceinline__ df2 df2_mul(f2x ahi, f2x nahi, f2x alo, const df2& x) {
    const f2x pn = mul2(nahi, x.hi);
    f2x e = fma2(ahi, x.hi, pn);
    e = fma2(ahi, x.lo, e);
    e = fma2(alo, x.hi, e);
    const f2x s = sub2(e, pn);
    return {s, sub2(e, add2(s, pn))};
}
__device__ __forceinline__ df2 df2_scale(const df2& x, float s) { return {mul2(x.hi, dup2(s)), mul2(x.lo, dup2(s))}; }

__device__ __forceinline__ f2x ld2(const float* p, size_t o) {
    return __ldg(reinterpret_cast<const unsigned long long*>(p + o));
}
// Row segment of a level: the hi and lo pairs at columns (x, x + 1) for x = i - 2, i, i + 2.
struct Row6 {
    df2 m, c, p;
};
__device__ __forceinline__ df2 ldp(const Level& L, size_t o) {
    return {ld2((const float*)L.hi, o), ld2((const float*)L.lo, o)};
}
__device__ __forceinline__ Row6 ld_row6(const Level& L, size_t o) { return {ldp(L, o - 2), ldp(L, o), ldp(L, o + 2)}; }

__device__ __forceinline__ df lane(const df2& v, int k) {
    float h0, h1, l0, l1;
    upk2(v.hi, h0, h1);
    upk2(v.lo, l0, l1);
    return k == 0 ? df{h0, l0} : df{h1, l1};
}
__device__ __forceinline__ df2 pack(const df& a, const df& b) { return {pk2(a.hi, b.hi), pk2(a.lo, b.lo)}; }

// The value at column offset d in -2 .. 3 from the pair's first node.
__device__ __forceinline__ df at(const Row6& r, int d) {
    return d < 0 ? lane(r.m, d + 2) : d < 2 ? lane(r.c, d) : lane(r.p, d - 2);
}

}  // namespace

// Block shape of k2_df2 (32 x kDf2BlockY threads).
constexpr int kDf2BlockY = 4;

// Thread (x, y) updates the node pair (i, i + 1), i = 2 (32 blockIdx.x + x),
// on K consecutive rows, walking down with the 2R + 1 rows of u^k
// around the current one in registers: each step loads one new row (row
// j + R + 1, issued before row j's arithmetic), so a thread reads each row of
// its walk once instead of 2R + 1 times.
template <int S, int BCM, int K>
__global__ void __launch_bounds__(32 * kDf2BlockY) k2_df2(Level cur, Level nxt, Geo g, Coef3<df> a, int gw) {
    constexpr int kDf2Rows = K;
    constexpr int R = (S == 13) ? 2 : 1;
    constexpr int W = 2 * R + 1;
    const int i0 = 2 * (blockIdx.x * 32 + threadIdx.x);
    const int j0 = (blockIdx.y * kDf2BlockY + threadIdx.y) * kDf2Rows;
    if (i0 >= g.nx || j0 >= g.ny) return;
    const bool two = i0 + 1 < g.nx;  // an odd row width leaves the last pair one node
    const size_t P = (size_t)g.pitch;
    size_t o = off(g, i0, j0);        // i0 + G even: 8-byte aligned pairs
    const f2x a10h = dup2(a.a10.hi), a10n = dup2(-a.a10.hi), a10l = dup2(a.a10.lo);
    const f2x a11h = dup2(a.a11.hi), a11n = dup2(-a.a11.hi), a11l = dup2(a.a11.lo);
    const f2x a20h = dup2(a.a20.hi), a20n = dup2(-a.a20.hi), a20l = dup2(a.a20.lo);
    Row6 win[W];  // rows j - R .. j + R of u^k (at most R + 1 rows past the grid: the ghost ring)
#pragma unroll
    for (int r = 0; r < W; ++r) win[r] = ld_row6(cur, (size_t)((ptrdiff_t)o + (ptrdiff_t)(r - R) * (ptrdiff_t)P));
#pragma unroll
    for (int k = 0; k < kDf2Rows; ++k) {
        const int j = j0 + k;
        if (j >= g.ny) break;
        Row6 ahead;
        if (k + 1 < kDf2Rows) ahead = ld_row6(cur, o + (size_t)(R + 1) * P);  // row j + R + 1
        const Row6& C = win[R];
        const Row6& N = win[R + 1];
        const Row6& Sr = win[R - 1];
        const df2 c = C.c;
        const df2 m4c = df2_scale(c, -4.0f);
        // class (1,0): (e + w) + (n + s), then -4 u_ij
        const df2 ew = pack(df_add(at(C, 1), at(C, -1)), df_add(at(C, 2), at(C, 0)));
        const df2 d10 = df2_add(df2_add(ew, df2_add(N.c, Sr.c)), m4c);
        df2 L = df2_mul(a10h, a10n, a10l, d10);
        if constexpr (S >= 9) {
            // class (1,1): (ne + sw) + (nw + se)
            const df2 nesw = pack(df_add(at(N, 1), at(Sr, -1)), df_add(at(N, 2), at(Sr, 0)));
            const df2 nwse = pack(df_add(at(N, -1), at(Sr, 1)), df_add(at(N, 0), at(Sr, 2)));
            const df2 d11 = df2_add(df2_add(nesw, nwse), m4c);
            L = df2_add(df2_mul(a11h, a11n, a11l, d11), L);
        }
        if constexpr (S == 13) {
            // class (2,0): (ee + ww) + (nn + ss)
            const df2 d20 = df2_add(df2_add(df2_add(C.p, C.m), df2_add(win[R + 2].c, win[R - 2].c)), m4c);
            L = df2_add(df2_mul(a20h, a20n, a20l, d20), L);
        }
        // u^{k-1} from the plane this thread overwrites with u^{k+1}: plain loads
        const df2 prev = {*reinterpret_cast<const unsigned long long*>((const float*)nxt.hi + o),
                          *reinterpret_cast<const unsigned long long*>((const float*)nxt.lo + o)};
        const df2 r = df2_add(df2_sub(df2_scale(c, 2.0f), prev), L);
        const df r0 = lane(r, 0), r1 = lane(r, 1);
        if (two) {
            *reinterpret_cast<unsigned long long*>((float*)nxt.hi + o) = r.hi;
            *reinterpret_cast<unsigned long long*>((float*)nxt.lo + o) = r.lo;
        } else {
            ((float*)nxt.hi)[o] = r0.hi;
            ((float*)nxt.lo)[o] = r0.lo;
        }
        if constexpr (BCM != BCM_ZERO) {
            write_images_bc<DT_F32X2, BCM>(nxt, g, i0, j, r0, gw);
            if (two) write_images_bc<DT_F32X2, BCM>(nxt, g, i0 + 1, j, r1, gw);
        }
#pragma unroll
        for (int r2 = 0; r2 + 1 < W; ++r2) win[r2] = win[r2 + 1];
        if (k + 1 < kDf2Rows) win[W - 1] = ahead;
        o += P;
    }
}

template <int S, int K>
static void launch_df2_sk(wave2d* h, const Coef3<df>& a) {
    const Level cur = h->level(h->cur), nxt = h->level(h->prv);
    const dim3 grid((((h->nx + 1) / 2) + 31) / 32, (h->ny + kDf2BlockY * K - 1) / (kDf2BlockY * K));
    const dim3 block(32, kDf2BlockY);
    switch (h->bc) {
        case WAVE2D_BC_PERIODIC:
            k2_df2<S, BCM_PERIODIC, K><<<grid, block, 0, h->stream>>>(cur, nxt, h->geo(), a, h->gw);
            break;
        case WAVE2D_BC_ODD:
            k2_df2<S, BCM_ODD, K><<<grid, block, 0, h->stream>>>(cur, nxt, h->geo(), a, h->gw);
            break;
        default:
            k2_df2<S, BCM_ZERO, K><<<grid, block, 0, h->stream>>>(cur, nxt, h->geo(), a, h->gw);
            break;
    }
}

// Rows per thread: the most of 4, 2 and 1 that still gives every SM 16 warps
// (a walk of 4 rows at 512^2 would leave most SMs without a warp).  Walks of
// 8 rows were measured slower (13-point 141 against 127.5 us at 4096^2): the
// unrolled body outgrows the instruction cache (ncu: no_instruction the top
// stall).
template <int S>
static void launch_df2_s(wave2d* h, const Coef3<df>& a) {
    const long long warps_x = (((long long)h->nx + 1) / 2 + 31) / 32;
    const long long want = 16LL * h->num_sms;
    auto warps = [&](int k) { return warps_x * (((long long)h->ny + k - 1) / k); };
    if (warps(4) >= want) launch_df2_sk<S, 4>(h, a);
    else if (warps(2) >= want) launch_df2_sk<S, 2>(h, a);
    else launch_df2_sk<S, 1>(h, a);
}

int df2_simple_step(wave2d* h, const Coef3<df>& a) {
    switch (h->scheme) {
        case 5: launch_df2_s<5>(h, a); break;
        case 9: launch_df2_s<9>(h, a); break;
        default: launch_df2_s<13>(h, a); break;
    }
    W2D_LAUNCHED("double-float two-step kernel launch");
    return WAVE2D_OK;
}

}  // namespace w2d
