// Launch of the derived-scheme TMA two-step kernel (kernels_chain.cuh).
#include "chain_launch.cuh"

namespace w2d {
using namespace chain_detail;
namespace {

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

template <typename T, int NC, int BCM, bool DIFF, bool DFORM>
int launch_tma(wave2d* h) {
    using Tile = ChainTile<T, NC>;
    constexpr int kNW = Tile::NW, kTH = Tile::TH;
    using C = ChainTmaCfg<T, NC, kTH, kNW>;
    auto kern = kc2_tma<T, NC, BCM, kTH, kNW, Tile::STAGES, Tile::MINB, DIFF, DFORM>;
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
    // difference form: the second staged box is d^k (plane dpl), updated in place
    const int second = DFORM ? h->dpl : h->prv;
    kern<<<grid, kNW * 32, smem, h->stream>>>(h->tm_cur[h->cur], h->tm_prev[second],
                                              reinterpret_cast<T*>(h->hi[h->prv]), h->geo(),
                                              coef_n<T, NC>(h->ca), tiles_x, n_tiles, h->gw, h->status,
                                              reinterpret_cast<T*>(h->hi[second]));
    W2D_LAUNCHED("derived-scheme TMA two-step kernel launch");
    return WAVE2D_OK;
}

}  // namespace

int chain_tma_step(wave2d* h) {
    int rc = WAVE2D_OK;
    dispatch_nc(h->nclass, [&](auto NCc) {
        constexpr int NC = decltype(NCc)::value;
        dispatch_bcm(h->bc, [&](auto Pc) {
            constexpr int P = decltype(Pc)::value;
            if (h->dtype == DT_F32) {
                if (h->diff_form) rc = launch_tma<float, NC, P, true, true>(h);
                else if (h->diff_sums) rc = launch_tma<float, NC, P, true, false>(h);
                else rc = launch_tma<float, NC, P, false, false>(h);
            } else {
                rc = h->diff_sums ? launch_tma<double, NC, P, true, false>(h) : launch_tma<double, NC, P, false, false>(h);
            }
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
