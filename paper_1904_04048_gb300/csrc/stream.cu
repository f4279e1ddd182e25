// Launches of the register-streaming temporal kernel (kernels_stream.cuh):
// one warp per strip of 128 columns and L rows, T two-steps per launch, out
// of place into the other pair of level planes.
#include <algorithm>

#include "kernels_stream.cuh"
#include "wave2d_impl.cuh"

namespace w2d {

// Periodic images of planes p and q in the first gw rings.
static int ring_images(wave2d* h, int p, int q) {
    // grid: x spans a band row, y = 2 gw band rows + the side-band blocks
    const int gx = std::min((h->nx + 2 * h->gw + 255) / 256, 16);
    const int side = std::max(1, std::min((h->ny * 2 * h->gw + 255) / 256 / gx, 64));
    k5_ring_images<<<dim3(gx, 2 * h->gw + side, 2), 256, 0, h->stream>>>(
        static_cast<float*>(h->hi[p]), static_cast<float*>(h->hi[q]), h->geo(), h->gw);
    W2D_LAUNCHED("periodic image kernel launch");
    return WAVE2D_OK;
}

template <int S, bool PER, int T, bool WRAP>
static int launch_stream_t(wave2d* h) {
    using C = StreamCfg<S, T>;
    auto kern = k5_stream<S, PER, T, WRAP>;
    constexpr int smem = stream_smem_bytes<S, T>();
    const int strips_x = (h->nx + C::OW - 1) / C::OW;
    const int L = h->temporal_oh;  // rows per strip
    const int strips_y = (h->ny + L - 1) / L;
    const int n = strips_x * strips_y;
    // the levels move to the other pair with their roles kept (plane p -> p ^ 2)
    const int oc = h->cur ^ 2, op = h->prv ^ 2;
    const Coef3<float> a{(float)h->a[0], (float)h->a[1], (float)h->a[2]};
    kern<<<(n + kStreamWarps - 1) / kStreamWarps, kStreamWarps * 32, smem, h->stream>>>(
        static_cast<const float*>(h->hi[h->cur]), static_cast<const float*>(h->hi[h->prv]),
        static_cast<float*>(h->hi[oc]), static_cast<float*>(h->hi[op]), h->geo(), a, strips_x, n, L);
    W2D_LAUNCHED("streaming temporal kernel launch");
    if constexpr (WRAP) {
        h->rings_stale = true;  // images rebuilt once before a ring reader runs
    } else if constexpr (PER) {
        int rc = ring_images(h, oc, op);
        if (rc != WAVE2D_OK) return rc;
    }
    h->cur = oc;
    h->prv = op;
    return WAVE2D_OK;
}

template <int S, bool PER, bool WRAP>
static int launch_stream_spw(wave2d* h) {
    switch (h->temporal_t) {
        case 2: return launch_stream_t<S, PER, 2, WRAP>(h);
        case 3: return launch_stream_t<S, PER, 3, WRAP>(h);
        case 6: return launch_stream_t<S, PER, 6, WRAP>(h);
        default: return launch_stream_t<S, PER, 4, WRAP>(h);
    }
}

// Periodic grids whose rows are whole vectors read their inputs at wrapped
// coordinates (WRAP); the others keep the ghost ring and a copy per launch.
template <int S, bool PER>
static int launch_stream_sp(wave2d* h) {
    if constexpr (PER) {
        if (h->nx % 4 == 0 && h->ny >= 16) return launch_stream_spw<S, PER, true>(h);
    }
    return launch_stream_spw<S, PER, false>(h);
}

template <int S>
static int launch_stream_s(wave2d* h) {
    return (h->bc == WAVE2D_BC_PERIODIC) ? launch_stream_sp<S, true>(h) : launch_stream_sp<S, false>(h);
}

int stream_fresh_rings(wave2d* h) {
    if (!h->rings_stale) return WAVE2D_OK;
    h->rings_stale = false;
    return ring_images(h, h->cur, h->prv);
}

int stream_launch(wave2d* h) {
    switch (h->scheme) {
        case 5: return launch_stream_s<5>(h);
        case 9: return launch_stream_s<9>(h);
        default: return launch_stream_s<13>(h);
    }
}

}  // namespace w2d
