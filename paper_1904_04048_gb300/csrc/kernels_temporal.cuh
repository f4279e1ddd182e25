// Temporally blocked two-step (Eq. A2 applied T times per HBM round trip).
//
// One CTA per output tile.  The CTA stages u^k and u^{k-1} on a region that
// extends the tile by T 16-byte vectors left and right and by R*T rows above
// and below, with one TMA box each, then advances the region T levels in
// shared memory: level t is computed on the region shrunk by one vector and R
// rows per side per level, in place over level t-2 (each node reads only its
// own older value), with one __syncthreads between levels.  The last two
// levels, u^{k+T} and u^{k+T-1}, are written for the tile only, to the other
// pair of level planes (other CTAs still read this tile's inputs as their
// halo).  Every node goes through two_step_update of stencil_ops.cuh, so T
// launches of this kernel equal T single steps bit for bit.
//
// Zero boundary: nodes outside the grid are forced to zero at every level
// (the ghost ring and the TMA out-of-bounds fill supply zero inputs).
// Periodic boundary: the inputs' ghost ring holds periodic images at least
// G >= max(4T, R T) nodes deep, written by every kernel in this mode.
#pragma once
#include "kernels.cuh"

namespace w2d {

template <int S, int RVW, int OH, int T>
struct TemporalCfg {
    static constexpr int R = (S == 13) ? 2 : 1;
    static constexpr int RW = 4 * RVW;       // region width (floats)
    static constexpr int OWV = RVW - 2 * T;  // output vectors per row
    static constexpr int OW = 4 * OWV;       // output width (floats)
    static constexpr int HY = R * T;         // halo rows per side
    static constexpr int RH = OH + 2 * HY;   // region rows
    static constexpr int BUF_BYTES = RW * RH * 4;
    static constexpr int WPR = RVW / 32;     // warps per region row
    static_assert(RVW % 32 == 0 && RW <= 256 && RH <= 256, "TMA box limit");
    static_assert(4 * T <= 16 && HY <= 16, "halo must fit the ghost ring");
};

struct Row4 {
    float a[8];  // x-2, x-1, x .. x+3, x+4, x+5
};

__device__ __forceinline__ Row4 smem_row4(const float* row, int lp_i, int v_i, int rp_i) {
    Row4 r;
    const float2 lp = *reinterpret_cast<const float2*>(row + lp_i);
    const float4 v = *reinterpret_cast<const float4*>(row + v_i);
    const float2 rp = *reinterpret_cast<const float2*>(row + rp_i);
    r.a[0] = lp.x; r.a[1] = lp.y;
    r.a[2] = v.x; r.a[3] = v.y; r.a[4] = v.z; r.a[5] = v.w;
    r.a[6] = rp.x; r.a[7] = rp.y;
    return r;
}

// Advance a staged region T levels in shared memory.  Q holds level k and P
// level k-1 on RH rows of 4*RVW floats whose column 0 is grid column gx0 and
// row 0 grid row gy0.  Level t is computed for region vectors [t, RVW-t) and
// rows [R t, RH - R t), in place over level t-2; the CTA synchronises after
// every level.  On return level k+T is in (T odd ? P : Q), level k+T-1 in the
// other buffer.  Zero boundary: nodes outside the grid are kept at zero.
template <int S, bool PER, int RVW, int T, int NW>
__device__ __forceinline__ void region_advance(float* Q, float* P, int RH, int gx0, int gy0, const Geo& g,
                                               const Coef3<float>& a) {
    constexpr int R = (S == 13) ? 2 : 1, RW = 4 * RVW, WPR = RVW / 32, NRG = NW / WPR;
    constexpr int UNROLL = (S == 13) ? 8 : 4;  // rows walked per unrolled step
    static_assert(NW % WPR == 0, "warps per row group");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int vidx = (warp % WPR) * 32 + lane;  // region vector owned by this thread
    const int rg = warp / WPR;                  // row group
    const int v_i = 4 * vidx;
    const int lp_i = max(v_i - 2, 0);           // clamped for lanes that never compute
    const int rp_i = min(v_i + 4, RW - 2);
    bool colin[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int gx = gx0 + v_i + e;
        colin[e] = gx >= 0 && gx < g.nx;
    }
    const f2x a10x2 = pk2(a.a10, a.a10), a11x2 = pk2(a.a11, a.a11), a20x2 = pk2(a.a20, a.a20);
#pragma unroll 1
    for (int t = 1; t <= T; ++t) {
        const float* src = (t & 1) ? Q : P;  // level k+t-1
        float* dst = (t & 1) ? P : Q;        // level k+t-2, overwritten by level k+t
        const bool active = vidx >= t && vidx < RVW - t;
        const int rlo = R * t, rhi = RH - R * t;
        const int per = (rhi - rlo + NRG - 1) / NRG;
        const int r0 = rlo + rg * per, r1 = min(r0 + per, rhi);
        if (active && r0 < r1) {
            Row4 win[2 * R + 1];
#pragma unroll
            for (int q = 1; q < 2 * R + 1; ++q) win[q] = smem_row4(src + (r0 - R + q - 1) * RW, lp_i, v_i, rp_i);
#pragma unroll UNROLL
            for (int r = r0; r < r1; ++r) {
#pragma unroll
                for (int q = 0; q < 2 * R; ++q) win[q] = win[q + 1];
                win[2 * R] = smem_row4(src + (r + R) * RW, lp_i, v_i, rp_i);
                float* dp = dst + r * RW + v_i;
                const float4 pv4 = *reinterpret_cast<const float4*>(dp);
                const float pv[4] = {pv4.x, pv4.y, pv4.z, pv4.w};
                float out[4];
                if constexpr (S == 5) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        Nbr<float> u;
                        u.c = win[R].a[e + 2];
                        u.e = win[R].a[e + 3];
                        u.w = win[R].a[e + 1];
                        u.n = win[R + 1].a[e + 2];
                        u.s = win[R - 1].a[e + 2];
                        out[e] = two_step_update<S>(u, pv[e], a);
                    }
                } else {
                    const float* up2 = win[R + 2 < 2 * R + 1 ? R + 2 : 2 * R].a;
                    const float* dn2 = win[R - 2 >= 0 ? R - 2 : 0].a;
#pragma unroll
                    for (int e = 0; e < 4; e += 2)
                        two_step_update_pair<S>(win[R].a, win[R + 1].a, win[R - 1].a, up2, dn2, e, pv[e],
                                                pv[e + 1], a10x2, a11x2, a20x2, out[e], out[e + 1]);
                }
                if constexpr (!PER) {
                    const int gy = gy0 + r;
                    const bool rowin = gy >= 0 && gy < g.ny;
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (!(rowin && colin[e])) out[e] = 0.0f;
                }
                *reinterpret_cast<float4*>(dp) = make_float4(out[0], out[1], out[2], out[3]);
            }
        }
        __syncthreads();
    }
}

struct Row2 {
    float a[6];  // x-2, x-1, x, x+1, x+2, x+3
};

__device__ __forceinline__ Row2 smem_row2(const float* row, int lp_i, int h_i, int rp_i) {
    Row2 r;
    const float2 lp = *reinterpret_cast<const float2*>(row + lp_i);
    const float2 v = *reinterpret_cast<const float2*>(row + h_i);
    const float2 rp = *reinterpret_cast<const float2*>(row + rp_i);
    r.a[0] = lp.x; r.a[1] = lp.y;
    r.a[2] = v.x; r.a[3] = v.y;
    r.a[4] = rp.x; r.a[5] = rp.y;
    return r;
}

// region_advance with two columns per lane: a region row is covered by
// 2 RVW / 32 warps, so the CTA splits the rows of a level among half as many
// row groups (fewer window prologues), and each row of the window is three
// 64-bit loads that consecutive lanes issue at an 8-byte stride (contiguous).
// Same levels, same nodes, same arithmetic as region_advance.
template <int S, bool PER, int RVW, int T, int NW>
__device__ __forceinline__ void region_advance2(float* Q, float* P, int RH, int gx0, int gy0, const Geo& g,
                                                const Coef3<float>& a) {
    constexpr int R = (S == 13) ? 2 : 1, RW = 4 * RVW, WPR = 2 * RVW / 32, NRG = NW / WPR;
    static_assert(NW % WPR == 0 && NRG >= 1, "warps per row group");
    constexpr int UNROLL = (S == 13) ? 8 : 4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int hidx = (warp % WPR) * 32 + lane;  // region column pair owned by this thread
    const int rg = warp / WPR;                  // row group
    const int h_i = 2 * hidx;
    const int lp_i = max(h_i - 2, 0);           // clamped for lanes that never compute
    const int rp_i = min(h_i + 2, RW - 2);
    bool colin[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int gx = gx0 + h_i + e;
        colin[e] = gx >= 0 && gx < g.nx;
    }
    const f2x a10x2 = pk2(a.a10, a.a10), a11x2 = pk2(a.a11, a.a11), a20x2 = pk2(a.a20, a.a20);
#pragma unroll 1
    for (int t = 1; t <= T; ++t) {
        const float* src = (t & 1) ? Q : P;  // level k+t-1
        float* dst = (t & 1) ? P : Q;        // level k+t-2, overwritten by level k+t
        const bool active = hidx >= 2 * t && hidx < 2 * RVW - 2 * t;  // vectors [t, RVW - t)
        const int rlo = R * t, rhi = RH - R * t;
        const int per = (rhi - rlo + NRG - 1) / NRG;
        const int r0 = rlo + rg * per, r1 = min(r0 + per, rhi);
        if (active && r0 < r1) {
            Row2 win[2 * R + 1];
#pragma unroll
            for (int q = 1; q < 2 * R + 1; ++q) win[q] = smem_row2(src + (r0 - R + q - 1) * RW, lp_i, h_i, rp_i);
#pragma unroll UNROLL
            for (int r = r0; r < r1; ++r) {
#pragma unroll
                for (int q = 0; q < 2 * R; ++q) win[q] = win[q + 1];
                win[2 * R] = smem_row2(src + (r + R) * RW, lp_i, h_i, rp_i);
                float* dp = dst + r * RW + h_i;
                const float2 pv2 = *reinterpret_cast<const float2*>(dp);
                float out[2];
                if constexpr (S == 5) {
                    const float pv[2] = {pv2.x, pv2.y};
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        Nbr<float> u;
                        u.c = win[R].a[e + 2];
                        u.e = win[R].a[e + 3];
                        u.w = win[R].a[e + 1];
                        u.n = win[R + 1].a[e + 2];
                        u.s = win[R - 1].a[e + 2];
                        out[e] = two_step_update<S>(u, pv[e], a);
                    }
                } else {
                    const float* up2 = win[R + 2 < 2 * R + 1 ? R + 2 : 2 * R].a;
                    const float* dn2 = win[R - 2 >= 0 ? R - 2 : 0].a;
                    two_step_update_pair<S>(win[R].a, win[R + 1].a, win[R - 1].a, up2, dn2, 0, pv2.x, pv2.y, a10x2,
                                            a11x2, a20x2, out[0], out[1]);
                }
                if constexpr (!PER) {
                    const int gy = gy0 + r;
                    const bool rowin = gy >= 0 && gy < g.ny;
#pragma unroll
                    for (int e = 0; e < 2; ++e)
                        if (!(rowin && colin[e])) out[e] = 0.0f;
                }
                *reinterpret_cast<float2*>(dp) = make_float2(out[0], out[1]);
            }
        }
        __syncthreads();
    }
}

// Write region rows [row0, row0 + OH) and vectors [vec0, vec0 + OWV) of the
// last two levels to the output planes (and their periodic images in the
// first gw rings when `edge`).
template <bool PER, int RVW, int NW>
__device__ __forceinline__ void region_store(const float* lastb, const float* otherb, int row0, int OH, int vec0,
                                             int OWV, int gx0, int gy0, const Geo& g, float* out_cur,
                                             float* out_prev, int gw, bool edge) {
    constexpr int RW = 4 * RVW, WPR = RVW / 32, NRG = NW / WPR;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int vidx = (warp % WPR) * 32 + lane;
    const int rg = warp / WPR;
    const int v_i = 4 * vidx;
    if (vidx < vec0 || vidx >= vec0 + OWV) return;
    const int gx = gx0 + v_i;
    const bool vec_images = (g.nx % 4 == 0) && g.nx >= 2 * gw && g.ny >= 2 * gw;
    const int per = (OH + NRG - 1) / NRG;
    const int r0 = row0 + rg * per, r1 = min(r0 + per, row0 + OH);
#pragma unroll 1
    for (int r = r0; r < r1; ++r) {
        const int gy = gy0 + r;
        if (gy >= g.ny || gx >= g.nx) break;
        const float4 vc = *reinterpret_cast<const float4*>(lastb + r * RW + v_i);
        const float4 vp = *reinterpret_cast<const float4*>(otherb + r * RW + v_i);
        const size_t o = off(g, gx, gy);
        if (gx + 4 <= g.nx) {
            *reinterpret_cast<float4*>(out_cur + o) = vc;
            *reinterpret_cast<float4*>(out_prev + o) = vp;
            if (PER && edge && vec_images) {
                store_vec_images(reinterpret_cast<float4*>(out_cur), g, gx, gy, vc, gw, 4);
                store_vec_images(reinterpret_cast<float4*>(out_prev), g, gx, gy, vp, gw, 4);
            }
        } else {
            const float c4[4] = {vc.x, vc.y, vc.z, vc.w}, p4[4] = {vp.x, vp.y, vp.z, vp.w};
            for (int e = 0; e < 4 && gx + e < g.nx; ++e) {
                out_cur[o + e] = c4[e];
                out_prev[o + e] = p4[e];
            }
        }
        if (PER && edge && !vec_images) {
            const Level Lc{out_cur, nullptr}, Lp{out_prev, nullptr};
            for (int e = 0; e < 4 && gx + e < g.nx; ++e) {
                write_images<DT_F32>(Lc, g, gx + e, gy, out_cur[o + e], gw);
                write_images<DT_F32>(Lp, g, gx + e, gy, out_prev[o + e], gw);
            }
        }
    }
}

template <int S, bool PER, int RVW, int OH, int T, int NW>
__global__ void __launch_bounds__(NW * 32, 1)
    k3_temporal(const __grid_constant__ CUtensorMap tm_cur, const __grid_constant__ CUtensorMap tm_prev,
                float* __restrict__ out_cur, float* __restrict__ out_prev, Geo g, Coef3<float> a,
                int tiles_x, int gw, int* status) {
    using C = TemporalCfg<S, RVW, OH, T>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    float* Q = reinterpret_cast<float*>(smem_raw + 1024);  // u^k
    float* P = Q + C::RW * C::RH;                          // u^{k-1}

    const int tid = threadIdx.x;
    const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    const int gx0 = tx * C::OW - 4 * T;  // grid column of region column 0
    const int gy0 = ty * OH - C::HY;     // grid row of region row 0

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, 2u * C::BUF_BYTES);
        tma_load_2d(Q, &tm_cur, bar, g.G + gx0, g.G + gy0);
        tma_load_2d(P, &tm_prev, bar, g.G + gx0, g.G + gy0);
    }
    const bool ok = mbar_wait_bounded(bar, 0, status);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) mbar_wait_bounded(bar, 0, status);  // drain the copies before exit
        return;
    }
    // radius-1 schemes walk two columns per lane (measured 4-5 % faster, the
    // shared-memory pipe being their limit); the 13-point scheme keeps four
    // (two independent packed pairs per lane, measured 2-3 % faster)
    if constexpr (S == 13) region_advance<S, PER, RVW, T, NW>(Q, P, C::RH, gx0, gy0, g, a);
    else region_advance2<S, PER, RVW, T, NW>(Q, P, C::RH, gx0, gy0, g, a);
    const bool edge = PER && (tx * C::OW < gw || tx * C::OW + C::OW > g.nx - gw || ty * OH < gw ||
                              ty * OH + OH > g.ny - gw);
    region_store<PER, RVW, NW>((T & 1) ? P : Q, (T & 1) ? Q : P, C::HY, OH, T, C::OWV, gx0, gy0, g, out_cur,
                               out_prev, gw, edge);
}

// Images in the first gw ghost rings, re-derived from the interior (used
// when a handle switches to a mode that reads a deeper ghost ring, and after
// raw state loads): periodic images, or the odd continuation's negated
// mirror images (zero on the boundary nodes).
template <int DT, int BCM>
__global__ void __launch_bounds__(256) k_refresh_ghosts(Level L, Geo g, int gw) {
    const int W = g.nx + 2 * gw, H = g.ny + 2 * gw;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)W * H;
         q += (long long)gridDim.x * blockDim.x) {
        const int ii = (int)(q % W) - gw, jj = (int)(q / W) - gw;
        if (ii >= 0 && ii < g.nx && jj >= 0 && jj < g.ny) continue;
        if constexpr (BCM == BCM_ODD) {
            double sign = 1.0;
            const int si = odd_index(ii, g.nx, sign), sj = odd_index(jj, g.ny, sign);
            if (si < 0 || sj < 0) {
                St<DT>::st(L, off(g, ii, jj), St<DT>::from_d(0.0));
            } else {
                const typename St<DT>::V v = St<DT>::ld(L, off(g, si, sj));
                St<DT>::st(L, off(g, ii, jj), sign < 0 ? vneg(v) : v);
            }
        } else {
            const int si = ((ii % g.nx) + g.nx) % g.nx, sj = ((jj % g.ny) + g.ny) % g.ny;
            St<DT>::st(L, off(g, ii, jj), St<DT>::ld(L, off(g, si, sj)));
        }
    }
}

}  // namespace w2d
