// Register-streaming temporally blocked two-step (Eq. A2 applied T times per
// HBM round trip; the levels live in registers, shared memory only stages the
// input rows).
//
// Each warp owns a strip of 128 grid columns (four consecutive nodes per
// lane) and L output rows, and walks down the strip one input row per step.
// The step that brings row rho of u^k in computes level t (t = 1..T) on row
// rho - tR, from the 2R+1 rows of level t-1 around it and row rho - tR of
// level t-2.  Every level keeps its last 2R+1 rows in registers, in a ring
// whose slots the unrolled loop addresses statically, so each node is read
// from HBM once, computed once per level and written once (levels k+T and
// k+T-1 to the other pair of planes).  Neighbours held by other lanes come by
// warp shuffles; the lanes at the warp edges compute HX >= R T halo columns
// that are never written, and the first 2RT rows of a strip only fill the
// rings (levels whose row is not yet valid are skipped).
//
// The per-node arithmetic is that of stencil_ops.cuh (two_step_update and
// two_step_update_pair with the same operands in the same order), so T levels
// of this kernel equal T single steps bit for bit.
//
// Zero boundary: nodes outside the grid are forced to zero at every level
// (their inputs come from the ghost ring, which holds zeros).  Periodic
// boundary: the kernel stores grid nodes only.  The WRAP variant (nx a
// multiple of 4, ny >= 16) reads its inputs at wrapped coordinates (a lane's
// 4-node vector wraps as a whole, rows wrap per step), so the ghost ring is
// neither read nor kept up to date between launches and k5_ring_images
// rebuilds the images once, before a kernel that reads the ring runs (the
// caller tracks this).  Otherwise the inputs' ghost ring holds periodic
// images at least R (T + 1) rows and HX columns deep and k5_ring_images
// copies them after every launch.  (Measured on GB300 at 4096^2: image
// stores inside the kernel made the 13-point level 23.0 us instead of 19.5
// with a copy per launch; wrapped reads with 64-row strips take it to 16.9,
// the copy kernel's 4.3-5.3 us per launch gone.)
#pragma once
#include <utility>

#include "kernels.cuh"

namespace w2d {

template <int S, int T>
struct StreamCfg {
    static constexpr int R = (S == 13) ? 2 : 1;
    static constexpr int D = R;                         // rows each level trails the one below
    static constexpr int WIN = 2 * D + 1;               // rows kept per level
    static constexpr int HX = (R * T + 3) / 4 * 4;      // halo columns per side
    static constexpr int OW = 128 - 2 * HX;             // output columns per strip
    static constexpr int HL = HX / 4;                   // halo lanes per side
    // Input row slots per warp in shared memory and rows copied ahead of the
    // step that uses them.  The 5- and 9-point kernels take a ring of 4 (2
    // rows ahead): their 72-108 registers would allow 5-7 CTAs per SM, and
    // the 8-slot ring's 32 KB per CTA held them to 6 (measured on GB300 at
    // 4096^2: 9-point T = 4 level 14.4 -> 13.4 us).  The 13-point kernel is
    // held to 4 CTAs per SM by its registers and keeps 8 slots, 6 ahead.
    static constexpr int NB = (S == 13) ? 8 : 4;
    static constexpr int PF = NB - 2;
    static_assert(R * T <= 16 && HX <= 16 && R * (T + 1) < 16, "halo must fit the ghost ring");
    static_assert(PF + 2 <= NB, "a slot is refilled two steps after its last read");
};

// Independent warps per CTA of the single-grid kernel: one.  The registers
// still hold 16 warps per SM (4 per scheduler partition), but single-warp
// CTAs are placed one warp at a time, so the SMs fill evenly (measured on
// GB300 at 4096^2: 13-point level 17.3 -> 17.0 us, difference form 23.5 ->
// 22.7; the 9-point kernel unchanged).  The batched kernel keeps CTAs of four
// warps.
constexpr int kStreamWarps = 1;
constexpr int kBatchStreamWarps = 4;
// shared memory per CTA of W warps: every warp's ring of input rows (both planes)
template <int S, int T, int W = kStreamWarps>
constexpr int stream_smem_bytes() {
    return W * StreamCfg<S, T>::NB * 2 * 32 * 16;
}

// 16-byte asynchronous copies global -> shared (cp.async, L2 only) and their
// completion waits.  The waits are hardware waits on this thread's own copies.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Two 16-byte global stores under one predicate (no branch, so the
// scheduler can overlap the steps of an unrolled group).
__device__ __forceinline__ void st2_pred(bool p, float* a, const float (&va)[4], float* b, const float (&vb)[4]) {
    asm volatile(
        "{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n"
        " @q st.global.v4.f32 [%1], {%3, %4, %5, %6};\n"
        " @q st.global.v4.f32 [%2], {%7, %8, %9, %10};\n}" ::"r"((int)p),
        "l"(a), "l"(b), "f"(va[0]), "f"(va[1]), "f"(va[2]), "f"(va[3]), "f"(vb[0]), "f"(vb[1]), "f"(vb[2]),
        "f"(vb[3])
        : "memory");
}

// Row of a lane in the layout of stencil_ops.cuh: v[k] = column x + k - 2 of
// the lane's vector at x.  NH columns on each side come from the neighbouring
// lanes (the lanes at the warp edges receive their own values: halo columns
// whose results are never stored).
template <int NH>
__device__ __forceinline__ void lane_row(const float (&own)[4], float (&v)[8]) {
    v[2] = own[0];
    v[3] = own[1];
    v[4] = own[2];
    v[5] = own[3];
    v[0] = v[1] = v[6] = v[7] = 0.0f;
    if constexpr (NH >= 1) {
        v[1] = __shfl_up_sync(0xffffffffu, own[3], 1);
        v[6] = __shfl_down_sync(0xffffffffu, own[0], 1);
    }
    if constexpr (NH >= 2) {
        v[0] = __shfl_up_sync(0xffffffffu, own[2], 1);
        v[7] = __shfl_down_sync(0xffffffffu, own[1], 1);
    }
}

// One level on one row: lv holds level t-1 (own columns) with the row of
// the updated node in slot CS and row r + d in slot (CS + d) mod WIN; prev is
// the node's row of level t-2.
template <int S, int WIN, int CS>
__device__ __forceinline__ void stream_level(const float (&lv)[WIN][4], const float (&prev)[4], float (&out)[4],
                                             const Coef3<float>& a, f2x a10x2, f2x a11x2, f2x a20x2) {
    constexpr int UP = (CS + 1) % WIN, DN = (CS + WIN - 1) % WIN;
    if constexpr (S == 5) {
        float c8[8];
        lane_row<1>(lv[CS], c8);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            Nbr<float> u;
            u.c = c8[e + 2];
            u.e = c8[e + 3];
            u.w = c8[e + 1];
            u.n = lv[UP][e];
            u.s = lv[DN][e];
            out[e] = two_step_update<S>(u, prev[e], a);
        }
    } else {
        constexpr int UP2 = (CS + 2) % WIN, DN2 = (CS + 2 * WIN - 2) % WIN;  // 13-point only
        float c8[8], up8[8], dn8[8], up28[8], dn28[8];
        lane_row<(S == 13) ? 2 : 1>(lv[CS], c8);
        lane_row<1>(lv[UP], up8);
        lane_row<1>(lv[DN], dn8);
        lane_row<0>(lv[S == 13 ? UP2 : UP], up28);  // the 9-point pair reads neither
        lane_row<0>(lv[S == 13 ? DN2 : DN], dn28);
#pragma unroll
        for (int e = 0; e < 4; e += 2)
            two_step_update_pair<S>(c8, up8, dn8, up28, dn28, e, prev[e], prev[e + 1], a10x2, a11x2, a20x2, out[e],
                                    out[e + 1]);
    }
}

// Storage and arithmetic modes of the streaming kernel.
constexpr int kStreamPlain = 0;  // u^k, u^{k-1}; sums of the nodes (stencil_ops.cuh)
constexpr int kStreamSums = 1;   // WAVE2D_DIFF_SUMS: u^k, u^{k-1}; sums of differences to the centre
constexpr int kStreamForm = 2;   // WAVE2D_DIFF_FORM: u^k, d^k = u^k - u^{k-1}; sums of differences

// Difference sums: one level on one row from the rows of u^{t-1} (as
// stream_level), every class sum formed from the differences to the centre,
// and the row `p` of the second input:
//   FORM (difference form): p = d^{t-1} = u^{t-1} - u^{t-2};
//     d^t = d^{t-1} + Lambda(u^{t-1}),  u^t = u^{t-1} + d^t;
//   otherwise: p = u^{t-2};  u^t = (2 u^{t-1} - u^{t-2}) + Lambda(u^{t-1}).
// The operations, their order and rounding are those of two_step_chain_dform
// and two_step_chain with difference sums (stencil_chain.cuh), lane by lane,
// so the results equal the one-level kernels of those modes bit for bit.
__device__ __forceinline__ float dsub(float x, float c) { return __fsub_rn(x, c); }

template <int S, int WIN, int CS, bool FORM>
__device__ __forceinline__ void stream_level_df(const float (&lv)[WIN][4], const float (&dprev)[4],
                                                float (&uout)[4], float (&dout)[4], const Coef3<float>& a,
                                                f2x a10x2, f2x a11x2, f2x a20x2) {
    constexpr int UP = (CS + 1) % WIN, DN = (CS + WIN - 1) % WIN;
    if constexpr (S == 5) {
        float c8[8];
        lane_row<1>(lv[CS], c8);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float c = c8[e + 2];
            const float s0 = __fadd_rn(__fadd_rn(dsub(c8[e + 3], c), dsub(c8[e + 1], c)),
                                       __fadd_rn(dsub(lv[UP][e], c), dsub(lv[DN][e], c)));
            const float L = __fmul_rn(a.a10, s0);
            if constexpr (FORM) {
                dout[e] = __fadd_rn(dprev[e], L);
                uout[e] = __fadd_rn(c, dout[e]);
            } else {
                uout[e] = __fadd_rn(__fmaf_rn(c, 2.0f, -dprev[e]), L);
            }
        }
    } else {
        constexpr int UP2 = (CS + 2) % WIN, DN2 = (CS + 2 * WIN - 2) % WIN;  // 13-point only
        float c[8], up[8], dn[8], up2[8], dn2[8];
        lane_row<(S == 13) ? 2 : 1>(lv[CS], c);
        lane_row<1>(lv[UP], up);
        lane_row<1>(lv[DN], dn);
        lane_row<0>(lv[S == 13 ? UP2 : UP], up2);
        lane_row<0>(lv[S == 13 ? DN2 : DN], dn2);
        const f2x m1 = pk2(-1.0f, -1.0f);
#pragma unroll
        for (int e = 0; e < 4; e += 2) {
            const f2x cc = pk2(c[e + 2], c[e + 3]);
            // pairs that start at an odd column: two scalar differences; even
            // pairs: x - c as one packed FMA x + c * (-1), the same rounding
            const f2x de = pk2(dsub(c[e + 3], c[e + 2]), dsub(c[e + 4], c[e + 3]));
            const f2x dw = pk2(dsub(c[e + 1], c[e + 2]), dsub(c[e + 2], c[e + 3]));
            const f2x dnn = fma2(cc, m1, pk2(up[e + 2], up[e + 3]));
            const f2x dss = fma2(cc, m1, pk2(dn[e + 2], dn[e + 3]));
            const f2x s0 = add2(add2(de, dw), add2(dnn, dss));
            f2x L = mul2(a10x2, s0);
            const f2x dne = pk2(dsub(up[e + 3], c[e + 2]), dsub(up[e + 4], c[e + 3]));
            const f2x dsw = pk2(dsub(dn[e + 1], c[e + 2]), dsub(dn[e + 2], c[e + 3]));
            const f2x dnw = pk2(dsub(up[e + 1], c[e + 2]), dsub(up[e + 2], c[e + 3]));
            const f2x dse = pk2(dsub(dn[e + 3], c[e + 2]), dsub(dn[e + 4], c[e + 3]));
            const f2x s1 = add2(add2(dne, dsw), add2(dnw, dse));
            L = fma2(a11x2, s1, L);
            if constexpr (S == 13) {
                const f2x dee = fma2(cc, m1, pk2(c[e + 4], c[e + 5]));
                const f2x dww = fma2(cc, m1, pk2(c[e], c[e + 1]));
                const f2x dn2n = fma2(cc, m1, pk2(up2[e + 2], up2[e + 3]));
                const f2x ds2s = fma2(cc, m1, pk2(dn2[e + 2], dn2[e + 3]));
                const f2x s2 = add2(add2(dee, dww), add2(dn2n, ds2s));
                L = fma2(a20x2, s2, L);
            }
            if constexpr (FORM) {
                const f2x dnew = add2(pk2(dprev[e], dprev[e + 1]), L);
                upk2(dnew, dout[e], dout[e + 1]);
                upk2(add2(cc, dnew), uout[e], uout[e + 1]);
            } else {  // 2c - p as one FMA, then + Lambda
                const f2x base = fma2(cc, pk2(2.0f, 2.0f), pk2(-dprev[e], -dprev[e + 1]));
                upk2(add2(base, L), uout[e], uout[e + 1]);
            }
        }
    }
}

template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
// f(std::integral_constant<int, i>) for i = 0 .. N-1, unrolled at compile time.
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

__device__ __forceinline__ void f4_to(const float4 v, float (&d)[4]) {
    d[0] = v.x;
    d[1] = v.y;
    d[2] = v.z;
    d[3] = v.w;
}

// Arguments of one warp's walk down its strip.
struct StreamWarp {
    const float* in_cur;
    const float* in_prev;
    float* out_cur;
    float* out_prev;
    float4* ring;     // this warp's input row slots: slot b, plane p at ring[(2 b + p) * 32]
    int lane, xl, xload, ymax, rho0, nsteps, ny;
    bool outlane, interior;
    bool colin[4];
};

// Stored row of input row y: clamped to the stored band (rows past it reach
// no stored node), or (WRAP) wrapped by selects.  Wrapped rows y >= 2 ny,
// which only strips taller than the grid reach and no stored node depends on,
// read row ny - 1.
template <bool WRAP>
__device__ __forceinline__ int stream_row(const StreamWarp& w, int y) {
    if constexpr (!WRAP) {
        return min(y, w.ymax);
    } else {
        const int r = y < 0 ? y + w.ny : y;  // y >= -R (T + 1) > -ny (ny >= 16 when wrapping)
        return r >= w.ny ? min(r - w.ny, w.ny - 1) : r;
    }
}

// Copy input step `step` (u^k row rho0 + step, u^{k-1} row rho0 + step - D)
// into its ring slot and close the copy group.
template <int D, int NB, bool WRAP>
__device__ __forceinline__ void stream_issue(const StreamWarp& w, const Geo& g, int step) {
    const int rho = w.rho0 + step;
    const int b = step % NB;
    float4* dst = w.ring + 2 * b * 32 + w.lane;
    cp_async16(smem_u32(dst), w.in_cur + off(g, w.xload, stream_row<WRAP>(w, rho)));
    cp_async16(smem_u32(dst + 32), w.in_prev + off(g, w.xload, stream_row<WRAP>(w, rho - D)));
    cp_async_commit();
}

// Stores of output row ro (levels k+T and k+T-1) with every check: partial
// vectors at the right edge, rows past the grid.
__device__ __forceinline__ void stream_store_checked(const StreamWarp& w, const Geo& g, int ro, const float (&top)[4],
                                                     const float (&pv)[4]) {
    if (!w.outlane || ro >= g.ny) return;
    const size_t o = off(g, w.xl, ro);
    const int xl = w.xl;
    if (xl + 4 <= g.nx) {
        *reinterpret_cast<float4*>(w.out_cur + o) = make_float4(top[0], top[1], top[2], top[3]);
        *reinterpret_cast<float4*>(w.out_prev + o) = make_float4(pv[0], pv[1], pv[2], pv[3]);
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (xl + e < g.nx) {
                w.out_cur[o + e] = top[e];
                w.out_prev[o + e] = pv[e];
            }
    }
}

// WIN consecutive steps from `base` (a multiple of WIN, so ring slots are
// static).  One body serves every step of every strip, so that the warps of
// an SM share one instruction stream: levels without valid inputs yet (the
// first T (D + R) steps) and steps past the end are skipped by warp-uniform
// branches, and interior strips (full vectors, rows inside the grid) store
// with predicated instructions.
template <int S, bool PER, int T, bool WRAP, int M>
__device__ __forceinline__ void stream_group(const StreamWarp& w, const Geo& g, const Coef3<float>& a, f2x a10x2,
                                             f2x a11x2, f2x a20x2, float (&q)[T][StreamCfg<S, T>::WIN][4],
                                             float (&qd)[T][StreamCfg<S, T>::WIN][4], int base) {
    using C = StreamCfg<S, T>;
    constexpr int R = C::R, D = C::D, WIN = C::WIN, NB = C::NB, PF = C::PF;
    constexpr bool DF = M == kStreamForm;
    static_for<WIN>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        const int step = base + s;
        if (step >= w.nsteps) return;
        const int rho = w.rho0 + step;
        cp_async_wait<PF - 1>();  // this step's copy group has landed
        const float4* src = w.ring + 2 * (step % NB) * 32 + w.lane;
        f4_to(src[0], q[0][s]);
        float pm[4];
        f4_to(src[32], pm);
        stream_issue<D, NB, WRAP>(w, g, step + PF);
        float top[4], dtop[4];  // level T on row rho - T D (and, difference form, its d)
        static_for<T>([&](auto tc) {
            constexpr int t = decltype(tc)::value + 1;
            constexpr int cs = ((s - t * D) % WIN + 2 * WIN) % WIN;  // slot of row rho - tD
            if (step < t * (D + R)) return;  // level t on row rho - tD has no valid inputs yet
            float out[4], dout[4];
            if constexpr (DF) {
                // the row's d^{t-1}: loaded with the step for t = 1, else kept
                // since level t-1 computed this row D steps ago
                if constexpr (t == 1) stream_level_df<S, WIN, cs, true>(q[0], pm, out, dout, a, a10x2, a11x2, a20x2);
                else stream_level_df<S, WIN, cs, true>(q[t - 1], qd[t >= 2 ? t - 1 : 0][cs], out, dout, a, a10x2,
                                                       a11x2, a20x2);
            } else if constexpr (M == kStreamSums) {
                if constexpr (t == 1) stream_level_df<S, WIN, cs, false>(q[0], pm, out, dout, a, a10x2, a11x2, a20x2);
                else stream_level_df<S, WIN, cs, false>(q[t - 1], q[t >= 2 ? t - 2 : 0][cs], out, dout, a, a10x2,
                                                        a11x2, a20x2);
            } else {
                if constexpr (t == 1) stream_level<S, WIN, cs>(q[0], pm, out, a, a10x2, a11x2, a20x2);
                else stream_level<S, WIN, cs>(q[t - 1], q[t >= 2 ? t - 2 : 0][cs], out, a, a10x2, a11x2, a20x2);
            }
            if constexpr (!PER) {
                const int r = rho - t * D;
                const bool rowin = r >= 0 && r < g.ny;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    out[e] = (rowin && w.colin[e]) ? out[e] : 0.0f;
                    if constexpr (DF) dout[e] = (rowin && w.colin[e]) ? dout[e] : 0.0f;
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if constexpr (t < T) {
                    q[t < T ? t : 0][cs][e] = out[e];
                    if constexpr (DF) qd[t < T ? t : 0][cs][e] = dout[e];
                } else {
                    top[e] = out[e];
                    if constexpr (DF) dtop[e] = dout[e];
                }
            }
        });
        if (step < T * (D + R)) return;  // no output row yet
        constexpr int ps = ((s - T * D) % WIN + 2 * WIN) % WIN;
        // second stored row: u^{k+T-1} of the row, or (difference form) d^{k+T}
        const float(&pv)[4] = DF ? dtop : q[T - 1][ps];
        const int ro = rho - T * D;  // in [y0, y0 + L)
        if (w.interior) {
            const size_t o = off(g, w.xl, ro);
            st2_pred(w.outlane, w.out_cur + o, top, w.out_prev + o, pv);
        } else {
            stream_store_checked(w, g, ro, top, pv);
        }
    });
}

// One warp's walk down strip `strip` of a grid: in_cur / in_prev are the
// planes of u^k and u^{k-1}; out_cur / out_prev receive u^{k+T} and
// u^{k+T-1}.  Strip s covers output columns [x0, x0 + OW) with
// x0 = (s % strips_x) OW and rows [y0, y0 + L) with y0 = (s / strips_x) L.
// ring: this warp's NB input row slots (both planes) in shared memory.
template <int S, bool PER, int T, bool WRAP, int M = kStreamPlain>
__device__ __forceinline__ void stream_strip(const float* __restrict__ in_cur, const float* __restrict__ in_prev,
                                             float* __restrict__ out_cur, float* __restrict__ out_prev,
                                             const Geo& g, const Coef3<float>& a, int strips_x, int strip, int L,
                                             float4* ring, int lane) {
    using C = StreamCfg<S, T>;
    constexpr int R = C::R, D = C::D, WIN = C::WIN, HX = C::HX, OW = C::OW, NB = C::NB, PF = C::PF;
    const int x0 = (strip % strips_x) * OW, y0 = (strip / strips_x) * L;
    StreamWarp w;
    w.in_cur = in_cur;
    w.in_prev = in_prev;
    w.out_cur = out_cur;
    w.out_prev = out_prev;
    w.ring = ring;
    w.lane = lane;
    w.xl = x0 - HX + 4 * lane;                  // grid column of the lane's first node (>= -G)
    w.xload = min(w.xl, g.pitch - g.G - 4);     // inside the row's storage; clamped lanes are
                                                // more than R T columns right of the grid
    w.ymax = g.ny + g.G - 1;                    // last stored row
    w.ny = g.ny;
    if constexpr (WRAP) w.xload = ((w.xl % g.nx) + g.nx) % g.nx;  // nx % 4 == 0: the vector stays whole
    w.rho0 = y0 - R * T;                        // first input row (>= -G)
    w.nsteps = L + T * (D + R);
#pragma unroll
    for (int e = 0; e < 4; ++e) w.colin[e] = w.xl + e >= 0 && w.xl + e < g.nx;
    w.outlane = lane >= C::HL && lane < 32 - C::HL && w.xl < g.nx;
    w.interior = x0 + OW <= g.nx && y0 + L <= g.ny;
    const f2x a10x2 = pk2(a.a10, a.a10), a11x2 = pk2(a.a11, a.a11), a20x2 = pk2(a.a20, a.a20);

    // q[t][slot][.]: level t (0 = u^k) at rows whose offset from rho0 is
    // congruent to slot modulo WIN
    float q[T][WIN][4];
    float qd[T][WIN][4];  // difference form: d^t rows of levels 1 .. T-1
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int s = 0; s < WIN; ++s)
#pragma unroll
            for (int e = 0; e < 4; ++e) q[t][s][e] = qd[t][s][e] = 0.0f;
#pragma unroll
    for (int s = 0; s < PF; ++s) stream_issue<D, NB, WRAP>(w, g, s);

#pragma unroll 1
    for (int base = 0; base < w.nsteps; base += WIN)
        stream_group<S, PER, T, WRAP, M>(w, g, a, a10x2, a11x2, a20x2, q, qd, base);
    cp_async_wait_all();  // no copy may land in shared memory after the warp exits
}

// One grid: warp (blockIdx.x * kStreamWarps + warp) walks strip of that
// index (strips_x strips across, n_strips in all).  M: kStreamPlain,
// kStreamSums or kStreamForm (difference form: in_prev holds d^k and
// out_prev receives d^{k+T}, rows read and written at the rows of u^k /
// u^{k+T}).
template <int S, bool PER, int T, bool WRAP, int M = kStreamPlain>
__global__ void __launch_bounds__(kStreamWarps * 32)
    k5_stream(const float* __restrict__ in_cur, const float* __restrict__ in_prev, float* __restrict__ out_cur,
              float* __restrict__ out_prev, Geo g, Coef3<float> a, int strips_x, int n_strips, int L) {
    constexpr int NB = StreamCfg<S, T>::NB;
    extern __shared__ float4 stream_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int strip = blockIdx.x * kStreamWarps + warp;
    if (strip >= n_strips) return;  // whole warps only; no copies issued yet
    stream_strip<S, PER, T, WRAP, M>(in_cur, in_prev, out_cur, out_prev, g, a, strips_x, strip, L,
                                      stream_smem + warp * NB * 2 * 32, lane);
}

// Periodic images of the two levels a streaming launch wrote, in the first gw
// rings, each ring cell copying the grid node it images.  Blocks with
// blockIdx.y < 2 gw copy one row of the top (y < gw) or bottom band over the
// ring's full width; the others copy the left and right bands, eight grid
// rows per 256 threads (2 gw = 32 cells per row).  blockIdx.z is the plane.
__device__ __forceinline__ int wrap_index(int i, int n) {
    if (i >= 0 && i < n) return i;
    if (i < 0 && i + n >= 0) return i + n;
    if (i >= n && i - n < n) return i - n;
    return ((i % n) + n) % n;  // grids narrower than the ring
}

static __global__ void __launch_bounds__(256) k5_ring_images(float* __restrict__ a, float* __restrict__ b, Geo g, int gw) {
    float* p = blockIdx.z ? b : a;
    const int t = threadIdx.x;
    if ((int)blockIdx.y < 2 * gw) {
        const int r = blockIdx.y;
        const int j = r < gw ? r - gw : g.ny + (r - gw);
        const int sj = wrap_index(j, g.ny);
        for (int i = (int)blockIdx.x * 256 + t - gw; i < g.nx + gw; i += gridDim.x * 256)
            p[off(g, i, j)] = p[off(g, wrap_index(i, g.nx), sj)];
    } else {
        const int rows_per_block = max(1, 256 / (2 * gw));  // gw <= 16 in every handle
        for (int base = ((int)blockIdx.y - 2 * gw) * gridDim.x + blockIdx.x; base * rows_per_block < g.ny;
             base += (gridDim.y - 2 * gw) * gridDim.x) {
            const int j = base * rows_per_block + t / (2 * gw), c = t % (2 * gw);
            if (j >= g.ny || t >= rows_per_block * 2 * gw) continue;
            const int i = c < gw ? c - gw : g.nx + (c - gw);
            p[off(g, i, j)] = p[off(g, wrap_index(i, g.nx), j)];
        }
    }
}

}  // namespace w2d
