// Launches of the derived-scheme kernels (kernels_chain.cuh) for a handle
// whose scheme is a prefix of nclass classes of the class chain.
#include <algorithm>

#include "kernels_chain.cuh"
#include "wave2d_impl.cuh"

namespace w2d {
namespace {

template <int V>
using IC = std::integral_constant<int, V>;
template <bool V>
using BC_ = std::integral_constant<bool, V>;

template <typename Fn>
void dispatch_nc(int nc, Fn&& fn) {
    switch (nc) {
        case 1: fn(IC<1>{}); break;
        case 2: fn(IC<2>{}); break;
        case 3: fn(IC<3>{}); break;
        case 4: fn(IC<4>{}); break;
        case 5: fn(IC<5>{}); break;
        case 6: fn(IC<6>{}); break;
        case 7: fn(IC<7>{}); break;
        default: fn(IC<8>{}); break;
    }
}
template <typename Fn>
void dispatch_dt(int dt, Fn&& fn) {
    switch (dt) {
        case DT_F64: fn(IC<DT_F64>{}); break;
        case DT_F32: fn(IC<DT_F32>{}); break;
        default: fn(IC<DT_F32X2>{}); break;
    }
}
template <typename Fn>
void dispatch_bool(bool v, Fn&& fn) {
    if (v) fn(BC_<true>{});
    else fn(BC_<false>{});
}

df split(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
template <typename V, int NC>
CoefN<V, NC> coef_n(const double* c, double scale = 1.0) {
    CoefN<V, NC> r;
    for (int q = 0; q < NC; ++q) {
        const double v = c[q] * scale;
        if constexpr (std::is_same<V, df>::value) r.a[q] = split(v);
        else r.a[q] = (V)v;
    }
    return r;
}

dim3 grid2d(const wave2d* h) { return dim3((h->nx + 31) / 32, (h->ny + 7) / 8); }

// Tile shape per storage type and class count: 8 warps on 32-row tiles,
// 3-stage pipeline, and at most 128 registers so that two CTAs share an SM
// (the window of 2R + 1 rows stays in registers without spilling for FP32 up
// to radius 4).  FP32 with eight classes (radius 4) keeps two stages so that
// two CTAs also fit in shared memory; FP64 with eight classes would spill
// under the cap and runs one CTA per SM.
template <typename T, int NC>
struct ChainTile {
    static constexpr bool F32 = sizeof(T) == 4;
    static constexpr int NW = 8;
    static constexpr int TH = 32;
    static constexpr int STAGES = (F32 && NC >= 8) ? 2 : 3;
    static constexpr int MINB = (!F32 && NC >= 8) ? 1 : 2;
};

template <typename T, int NC, bool PER>
int launch_tma(wave2d* h) {
    using Tile = ChainTile<T, NC>;
    constexpr int kNW = Tile::NW, kTH = Tile::TH;
    using C = ChainTmaCfg<T, NC, kTH, kNW>;
    auto kern = kc2_tma<T, NC, PER, kTH, kNW, Tile::STAGES, Tile::MINB>;
    const int smem = 2048 + Tile::STAGES * C::STAGE_BYTES;
    static thread_local int configured_smem = -1;  // per instantiation
    if (configured_smem != smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(derived-scheme TMA kernel)");
        configured_smem = smem;
    }
    static thread_local int occ = 0;
    if (occ == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kNW * 32, smem);
        if (e != cudaSuccess || occ < 1) occ = 1;
    }
    const int tiles_x = (h->nx + C::TW - 1) / C::TW;
    const int tiles_y = (h->ny + kTH - 1) / kTH;
    const int n_tiles = tiles_x * tiles_y;
    int per_sm = h->tune.ctas_per_sm;
    if (per_sm <= 0) per_sm = (2.0 * (double)h->plane_bytes <= 1.25 * (double)h->l2_bytes) ? occ : 1;
    per_sm = std::max(1, std::min(per_sm, occ));
    const int grid = std::min(n_tiles, per_sm * h->num_sms);
    kern<<<grid, kNW * 32, smem, h->stream>>>(h->tm_cur[h->cur], h->tm_prev[h->prv],
                                              reinterpret_cast<T*>(h->hi[h->prv]), h->geo(),
                                              coef_n<T, NC>(h->ca), tiles_x, n_tiles, h->gw, h->status);
    W2D_LAUNCHED("derived-scheme TMA two-step kernel launch");
    return WAVE2D_OK;
}

}  // namespace

int chain_first_step(wave2d* h, const double* du0, const double* dv0, const ExactTab& ex, const Reduce& rd) {
    const Level L0 = h->level(1), L1 = h->level(0);  // u^0 -> plane 1 (u^{k-1}), u^1 -> plane 0
    dispatch_dt(h->dtype, [&](auto DTc) {
        dispatch_nc(h->nclass, [&](auto NCc) {
            constexpr int NC = decltype(NCc)::value;
            const CoefN<double, NC> ahalf = coef_n<double, NC>(h->ca, 0.5), b = coef_n<double, NC>(h->cb);
            dispatch_bool(h->bc == WAVE2D_BC_PERIODIC, [&](auto Pc) {
                dispatch_bool(h->tracking, [&](auto Tc) {
                    kc1_first_step<decltype(DTc)::value, NC, decltype(Pc)::value, decltype(Tc)::value>
                        <<<grid2d(h), dim3(32, 8), 0, h->stream>>>(du0, dv0, L0, L1, h->geo(), ahalf, b, h->tau,
                                                                   ex, rd, h->gw);
                });
            });
        });
    });
    W2D_LAUNCHED("derived-scheme first-step kernel launch");
    return WAVE2D_OK;
}

int chain_simple_step(wave2d* h, bool track, const ExactTab& ex, const Reduce& rd) {
    const Level cur = h->level(h->cur), nxt = h->level(h->prv);
    dispatch_dt(h->dtype, [&](auto DTc) {
        constexpr int DT = decltype(DTc)::value;
        using V = typename St<DT>::V;
        dispatch_nc(h->nclass, [&](auto NCc) {
            constexpr int NC = decltype(NCc)::value;
            const CoefN<V, NC> a = coef_n<V, NC>(h->ca);
            dispatch_bool(h->bc == WAVE2D_BC_PERIODIC, [&](auto Pc) {
                dispatch_bool(track, [&](auto Tc) {
                    kc2_simple<DT, NC, decltype(Pc)::value, decltype(Tc)::value>
                        <<<grid2d(h), dim3(32, 8), 0, h->stream>>>(cur, nxt, h->geo(), a, ex, rd, h->gw);
                });
            });
        });
    });
    W2D_LAUNCHED("derived-scheme two-step kernel launch");
    return WAVE2D_OK;
}

int chain_tma_step(wave2d* h) {
    int rc = WAVE2D_OK;
    dispatch_nc(h->nclass, [&](auto NCc) {
        constexpr int NC = decltype(NCc)::value;
        dispatch_bool(h->bc == WAVE2D_BC_PERIODIC, [&](auto Pc) {
            constexpr bool P = decltype(Pc)::value;
            rc = (h->dtype == DT_F32) ? launch_tma<float, NC, P>(h) : launch_tma<double, NC, P>(h);
        });
    });
    return rc;
}

void chain_tma_box(const wave2d* h, int& box_w, int& box_h, int& tile_w, int& tile_h) {
    dispatch_nc(h->nclass, [&](auto NCc) {
        constexpr int NC = decltype(NCc)::value;
        if (h->dtype == DT_F32) {
            using Tile = ChainTile<float, NC>;
            using C = ChainTmaCfg<float, NC, Tile::TH, Tile::NW>;
            box_w = C::BOX_W, box_h = C::BOX_H, tile_w = C::TW, tile_h = Tile::TH;
        } else {
            using Tile = ChainTile<double, NC>;
            using C = ChainTmaCfg<double, NC, Tile::TH, Tile::NW>;
            box_w = C::BOX_W, box_h = C::BOX_H, tile_w = C::TW, tile_h = Tile::TH;
        }
    });
}

}  // namespace w2d
