// Kernels of the derived schemes (a prefix of NC classes of the class chain,
// stencil radius up to 4): the same three kernels as for the Section 6
// schemes, with the node arithmetic of stencil_chain.cuh.
//
//   kc1_first_step  first time step, Eq. A1, FP64 math, one node per thread
//   kc2_simple      two-step, Eq. A2, one node per thread (any storage type),
//                   optional fused space-time error reduction
//   (the two-step kernels also come with the difference sums of
//   stencil_chain.cuh, DIFF = true, for FP32 and FP64 storage)
//   kc2_tma         two-step through TMA-staged tiles (F32 / F64 storage):
//                   persistent CTAs, NSTAGES-deep mbarrier pipeline, each lane
//                   walks down one column vector keeping 2R + 1 rows in
//                   registers
//
// Level planes, ghost rings and periodic images are those of kernels.cuh
// (ghost ring G = 16 >= R, images kept in the first gw = R rings).
#pragma once
#include "kernels.cuh"
#include "stencil_chain.cuh"

namespace w2d {

// DFORM: L0 receives d^1 = u^1 - u^0 (formed in FP64) instead of u^0.
template <int DT, int NC, int BCM, bool TRACK, bool DFORM>
__global__ void __launch_bounds__(256) kc1_first_step(const double* __restrict__ u0,
                                                      const double* __restrict__ v0, Level L0,
                                                      Level L1, Geo g, CoefN<double, NC> ahalf,
                                                      CoefN<double, NC> b, double tau, ExactTab ex,
                                                      Reduce rd, int gw) {
    using T = St<DT>;
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    double s0 = 0, s1 = 0, m0 = 0, m1 = 0;
    if (i < g.nx && j < g.ny) {
        const auto u = [&](int dx, int dy) { return fetch_bc(u0, g.nx, g.ny, BCM, i + dx, j + dy); };
        const auto v = [&](int dx, int dy) { return fetch_bc(v0, g.nx, g.ny, BCM, i + dx, j + dy); };
        const double uc = u(0, 0), vc = v(0, 0);
        const double u1 = first_step_chain<NC>(u, v, uc, vc, ahalf, b, tau);
        const size_t o = off(g, i, j);
        const typename T::V q0 = T::from_d(DFORM ? __dsub_rn(u1, uc) : uc), q1 = T::from_d(u1);
        T::st(L0, o, q0);
        T::st(L1, o, q1);
        if (BCM != BCM_ZERO) {
            if (!DFORM) write_images_bc<DT, BCM>(L0, g, i, j, q0, gw);  // d is read at its own node only
            write_images_bc<DT, BCM>(L1, g, i, j, q1, gw);
        }
        if (TRACK) error_terms(T::to_d(q1), exact_at(ex, i, j), s0, s1, m0, m1, rd.status);
    }
    if (TRACK) reduce_finalize<256>(s0, s1, m0, m1, rd);
}

// DFORM: `nxt` receives u^{k+1}; `dpl` holds d^k and receives d^{k+1} in place.
template <int DT, int NC, int BCM, bool TRACK, bool DIFF, bool DFORM>
__global__ void __launch_bounds__(256) kc2_simple(Level cur, Level nxt, Geo g,
                                                  CoefN<typename St<DT>::V, NC> a, ExactTab ex,
                                                  Reduce rd, int gw, Level dpl) {
    using T = St<DT>;
    using V = typename T::V;
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    double s0 = 0, s1 = 0, m0 = 0, m1 = 0;
    if (i < g.nx && j < g.ny) {
        const size_t o = off(g, i, j);
        const long long P = g.pitch;
        const auto u = [&](int dx, int dy) { return T::ldg(cur, (size_t)((long long)o + dy * P + dx)); };
        V r;
        if constexpr (DFORM) {
            V dn;
            two_step_chain_dform<NC, DIFF>(u, u(0, 0), T::ld(dpl, o), a, r, dn);
            T::st(dpl, o, dn);
        } else {
            r = two_step_chain<NC, DIFF>(u, u(0, 0), T::ld(nxt, o), a);
        }
        T::st(nxt, o, r);
        if (BCM != BCM_ZERO) write_images_bc<DT, BCM>(nxt, g, i, j, r, gw);
        if (TRACK) error_terms(T::to_d(r), exact_at(ex, i, j), s0, s1, m0, m1, rd.status);
    }
    if (TRACK) reduce_finalize<256>(s0, s1, m0, m1, rd);
}

// ---------------------------------------------------------------------------
// TMA tiles.  Box of u^k: TW + 2 HB columns (HB = halo columns, a whole
// number of vectors >= R) by TH + 2R rows; box of u^{k-1}: TW x TH.  A lane's
// row buffer holds columns x - H .. x + VEC - 1 + H of one row (H = 2 for
// R <= 2, else 4).
// ---------------------------------------------------------------------------
template <typename T, int NC, int TH, int NW>
struct ChainTmaCfg {
    static constexpr int VEC = TmaVec<T>::N;
    static constexpr int R = chain_radius(NC);
    static constexpr int H = R <= 2 ? 2 : 4;
    static constexpr int HB = (H + VEC - 1) / VEC * VEC;
    static constexpr int TW = 32 * VEC;
    static constexpr int BOX_W = TW + 2 * HB;
    static constexpr int BOX_H = TH + 2 * R;
    static constexpr int CUR_BYTES = ((BOX_W * BOX_H * (int)sizeof(T)) + 127) / 128 * 128;
    static constexpr int PREV_BYTES = ((TW * TH * (int)sizeof(T)) + 127) / 128 * 128;
    static constexpr int STAGE_BYTES = CUR_BYTES + PREV_BYTES;
    static constexpr int RPW = TH / NW;
    static_assert(TH % NW == 0, "rows per warp");
    static_assert(BOX_W <= 256 && BOX_H <= 256, "TMA box limit");
    static_assert(R <= 4 && H >= R && HB >= H, "halo");
};

template <typename T, int VEC, int H>
struct ChainRow {
    T a[VEC + 2 * H];  // columns x - H .. x + VEC - 1 + H
};

// Row buffer of the lane whose vector starts at column `col` of a staged row
// (col - H is 8-byte aligned for F32 with H = 2, 16-byte aligned otherwise).
template <typename T, int VEC, int H>
__device__ __forceinline__ ChainRow<T, VEC, H> chain_load_row(const T* row, int col) {
    ChainRow<T, VEC, H> r;
    const T* p = row + col - H;
    if constexpr (sizeof(T) == 4 && H == 2) {
        const float2 lp = *reinterpret_cast<const float2*>(p);
        const float4 v = *reinterpret_cast<const float4*>(p + 2);
        const float2 rp = *reinterpret_cast<const float2*>(p + 6);
        r.a[0] = lp.x; r.a[1] = lp.y;
        r.a[2] = v.x; r.a[3] = v.y; r.a[4] = v.z; r.a[5] = v.w;
        r.a[6] = rp.x; r.a[7] = rp.y;
    } else if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < (VEC + 2 * H) / 4; ++q) {
            const float4 v = *reinterpret_cast<const float4*>(p + 4 * q);
            r.a[4 * q] = v.x; r.a[4 * q + 1] = v.y; r.a[4 * q + 2] = v.z; r.a[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < (VEC + 2 * H) / 2; ++q) {
            const double2 v = *reinterpret_cast<const double2*>(p + 2 * q);
            r.a[2 * q] = v.x; r.a[2 * q + 1] = v.y;
        }
    }
    return r;
}

// DFORM: tm_prev stages d^k; u^{k+1} goes to `nxt`, d^{k+1} to `dout` (in
// place over d^k, which this tile has already staged).
template <typename T, int NC, int BCM, int TH, int NW, int NSTAGES, int MINB, bool DIFF, bool DFORM>
__global__ void __launch_bounds__(NW * 32, MINB)
    kc2_tma(const __grid_constant__ CUtensorMap tm_cur, const __grid_constant__ CUtensorMap tm_prev,
            T* __restrict__ nxt, Geo g, CoefN<T, NC> a, int tiles_x, int n_tiles, int gw, int* status,
            T* __restrict__ dout) {
    using C = ChainTmaCfg<T, NC, TH, NW>;
    constexpr int VEC = C::VEC, R = C::R, H = C::H, HB = C::HB, TW = C::TW, BOX_W = C::BOX_W,
                  RPW = C::RPW;
    constexpr int DT = sizeof(T) == 4 ? DT_F32 : DT_F64;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    unsigned char* stages = smem_raw + 1024;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < NSTAGES; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
        fence_proxy_async_smem();
        abort_flag = 0;
    }
    __syncthreads();

    auto issue = [&](int t, int s) {
        const int tx = t % tiles_x, ty = t / tiles_x;
        unsigned char* st = stages + (size_t)s * C::STAGE_BYTES;
        mbar_arrive_expect_tx(&bars[s], (unsigned)(BOX_W * C::BOX_H * sizeof(T) + TW * TH * sizeof(T)));
        tma_load_2d(st, &tm_cur, &bars[s], g.G + tx * TW - HB, g.G + ty * TH - R);
        tma_load_2d(st + C::CUR_BYTES, &tm_prev, &bars[s], g.G + tx * TW, g.G + ty * TH);
    };

    const int stride = gridDim.x;
    if (tid == 0) {
        for (int s = 0; s < NSTAGES; ++s) {
            const int t = blockIdx.x + s * stride;
            if (t < n_tiles) issue(t, s);
        }
    }

    int it = 0;
    for (int t = blockIdx.x; t < n_tiles; t += stride, ++it) {
        const int s = it % NSTAGES;
        const unsigned parity = (unsigned)(it / NSTAGES) & 1u;
        const bool ok = mbar_wait_bounded(&bars[s], parity, status);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) abort_flag = 1;
            break;
        }
        const T* cur_s = reinterpret_cast<const T*>(stages + (size_t)s * C::STAGE_BYTES);
        const T* prev_s = reinterpret_cast<const T*>(stages + (size_t)s * C::STAGE_BYTES + C::CUR_BYTES);
        const int tx = t % tiles_x, ty = t / tiles_x;
        const int x = tx * TW + lane * VEC;
        const int r0 = warp * RPW;
        const int col = HB + lane * VEC;  // this lane's vector inside a staged row
        const bool edge = BCM != BCM_ZERO && (tx * TW < gw || tx * TW + TW > g.nx - gw || ty * TH < gw ||
                                              ty * TH + TH > g.ny - gw);
        const bool vec_images = BCM == BCM_PERIODIC && (g.nx % VEC == 0) && g.nx >= 2 * gw && g.ny >= 2 * gw;

        // win[q] holds staged row (r + q) of u^k, i.e. grid row y - R + q
        ChainRow<T, VEC, H> win[2 * R + 1];
#pragma unroll
        for (int q = 1; q < 2 * R + 1; ++q) win[q] = chain_load_row<T, VEC, H>(cur_s + (r0 + q - 1) * BOX_W, col);
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
#pragma unroll
            for (int q = 0; q < 2 * R; ++q) win[q] = win[q + 1];
            win[2 * R] = chain_load_row<T, VEC, H>(cur_s + (r0 + r + 2 * R) * BOX_W, col);
            T pv[VEC];
            if constexpr (VEC == 4) {
                const float4 p = *reinterpret_cast<const float4*>(prev_s + (r0 + r) * TW + lane * 4);
                pv[0] = p.x; pv[1] = p.y; pv[2] = p.z; pv[3] = p.w;
            } else {
                const double2 p = *reinterpret_cast<const double2*>(prev_s + (r0 + r) * TW + lane * 2);
                pv[0] = p.x; pv[1] = p.y;
            }
            T out[VEC], dnew[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const auto u = [&](int dx, int dy) -> T { return win[R + dy].a[H + e + dx]; };
                if constexpr (DFORM) two_step_chain_dform<NC, DIFF>(u, u(0, 0), pv[e], a, out[e], dnew[e]);
                else out[e] = two_step_chain<NC, DIFF>(u, u(0, 0), pv[e], a);
            }
            const int y = ty * TH + r0 + r;
            if (y < g.ny) {
                T* gp = nxt + off(g, x, y);
                if constexpr (DFORM) {
                    T* dp = dout + off(g, x, y);
                    if (x + VEC <= g.nx) {
                        if constexpr (VEC == 4)
                            *reinterpret_cast<float4*>(dp) = make_float4(dnew[0], dnew[1], dnew[2], dnew[3]);
                        else
                            *reinterpret_cast<double2*>(dp) = make_double2(dnew[0], dnew[1]);
                    } else {
#pragma unroll
                        for (int e = 0; e < VEC; ++e)
                            if (x + e < g.nx) dp[e] = dnew[e];
                    }
                }
                if (x + VEC <= g.nx) {
                    if constexpr (VEC == 4) {
                        const float4 v = make_float4(out[0], out[1], out[2], out[3]);
                        *reinterpret_cast<float4*>(gp) = v;
                        if (edge && vec_images) store_vec_images(reinterpret_cast<float4*>(nxt), g, x, y, v, gw, 4);
                    } else {
                        const double2 v = make_double2(out[0], out[1]);
                        *reinterpret_cast<double2*>(gp) = v;
                        if (edge && vec_images) store_vec_images(reinterpret_cast<double2*>(nxt), g, x, y, v, gw, 2);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e)
                        if (x + e < g.nx) gp[e] = out[e];
                }
            }
        }
        if (edge && !vec_images) {
            const Level L{nxt, nullptr};
#pragma unroll 1
            for (int r = 0; r < RPW; ++r) {
                const int y = ty * TH + r0 + r;
                if (y >= g.ny) break;
#pragma unroll 1
                for (int e = 0; e < VEC; ++e)
                    if (x + e < g.nx) write_images_bc<DT, BCM>(L, g, x + e, y, nxt[off(g, x + e, y)], gw);
            }
        }
        __syncthreads();  // every warp is done with stage s
        if (tid == 0) {
            const int tn = t + NSTAGES * stride;
            if (tn < n_tiles) issue(tn, s);
        }
    }

    if (abort_flag && tid == 0) {
        int it2 = it;
        for (int t = blockIdx.x + it * stride; t < n_tiles && it2 < it + NSTAGES; t += stride, ++it2)
            mbar_wait_bounded(&bars[it2 % NSTAGES], (unsigned)(it2 / NSTAGES) & 1u, status);
    }
}

}  // namespace w2d
