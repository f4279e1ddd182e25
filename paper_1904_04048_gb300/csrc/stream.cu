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

template <int S, bool PER, int T, bool WRAP, int M>
static int launch_stream_t(wave2d* h) {
    using C = StreamCfg<S, T>;
    constexpr bool DF = M == kStreamForm;
    auto kern = k5_stream<S, PER, T, WRAP, M>;
    constexpr int smem = stream_smem_bytes<S, T>();
    const int strips_x = (h->nx + C::OW - 1) / C::OW;
    const int L = h->temporal_oh;  // rows per strip
    const int strips_y = (h->ny + L - 1) / L;
    const int n = strips_x * strips_y;
    // Plain: the levels move to the other pair with their roles kept (plane
    // p -> p ^ 2).  Difference form: u^k (cur) -> u^{k+T} in the other u plane
    // (prv), d^k (dpl) -> d^{k+T} in the other d plane (dpl ^ 1).
    const int ic = h->cur, ip = DF ? h->dpl : h->prv;
    const int oc = DF ? h->prv : (h->cur ^ 2), op = DF ? (h->dpl ^ 1) : (h->prv ^ 2);
    // class-chain handles (difference sums or form, derived schemes) carry
    // the class coefficients: the Section 6 scheme's, or a derived scheme's
    // first one to three classes
    const double* ad = h->nclass > 0 ? h->ca : h->a;
    const Coef3<float> a{(float)ad[0], (float)ad[1], (float)ad[2]};
    kern<<<(n + kStreamWarps - 1) / kStreamWarps, kStreamWarps * 32, smem, h->stream>>>(
        static_cast<const float*>(h->hi[ic]), static_cast<const float*>(h->hi[ip]), static_cast<float*>(h->hi[oc]),
        static_cast<float*>(h->hi[op]), h->geo(), a, strips_x, n, L);
    W2D_LAUNCHED("streaming temporal kernel launch");
    if constexpr (WRAP) {
        h->rings_stale = true;  // images rebuilt once before a ring reader runs
    } else if constexpr (PER) {
        static_assert(!DF, "periodic difference-form streaming reads wrapped coordinates");
        int rc = ring_images(h, oc, op);
        if (rc != WAVE2D_OK) return rc;
    }
    if constexpr (DF) {
        std::swap(h->cur, h->prv);
        h->dpl ^= 1;
    } else {
        h->cur = oc;
        h->prv = op;
    }
    return WAVE2D_OK;
}

template <int S, bool PER, bool WRAP, int M>
static int launch_stream_spw(wave2d* h) {
    if constexpr (M == kStreamForm) {  // depths 2..4 (the d rows take registers)
        switch (h->temporal_t) {
            case 2: return launch_stream_t<S, PER, 2, WRAP, M>(h);
            case 3: return launch_stream_t<S, PER, 3, WRAP, M>(h);
            default: return launch_stream_t<S, PER, 4, WRAP, M>(h);
        }
    } else {
        switch (h->temporal_t) {
            case 2: return launch_stream_t<S, PER, 2, WRAP, M>(h);
            case 3: return launch_stream_t<S, PER, 3, WRAP, M>(h);
            case 6: return launch_stream_t<S, PER, 6, WRAP, M>(h);
            default: return launch_stream_t<S, PER, 4, WRAP, M>(h);
        }
    }
}

// Periodic grids whose rows are whole vectors read their inputs at wrapped
// coordinates (WRAP); the others keep the ghost ring and a copy per launch.
// The difference form reads d^k at the halo lanes' own nodes, whose ring
// images nothing keeps: periodic difference-form handles stream only with
// wrapped reads (the kernel choice ensures it).
template <int S, bool PER, int M>
static int launch_stream_sp(wave2d* h) {
    if constexpr (PER) {
        if (h->nx % 4 == 0 && h->ny >= 16) return launch_stream_spw<S, PER, true, M>(h);
        if constexpr (M == kStreamForm)
            return set_error(WAVE2D_ERR_ARG, "periodic difference-form streaming needs nx %% 4 == 0, ny >= 16");
        else
            return launch_stream_spw<S, PER, false, M>(h);
    } else {
        return launch_stream_spw<S, PER, false, M>(h);
    }
}

template <int S, int M>
static int launch_stream_sm(wave2d* h) {
    return h->bc == WAVE2D_BC_PERIODIC ? launch_stream_sp<S, true, M>(h) : launch_stream_sp<S, false, M>(h);
}

template <int S>
static int launch_stream_s(wave2d* h) {
    if (h->diff_form) return launch_stream_sm<S, kStreamForm>(h);
    if (h->nclass > 0 && h->diff_sums) return launch_stream_sm<S, kStreamSums>(h);
    return launch_stream_sm<S, kStreamPlain>(h);
}

int stream_fresh_rings(wave2d* h) {
    if (!h->rings_stale) return WAVE2D_OK;
    h->rings_stale = false;
    return ring_images(h, h->cur, h->prv);
}

int stream_launch(wave2d* h) {
    // the kernel writes out of place: both pairs of level planes must exist
    if (h->nlevels < 4 || h->dtype != WAVE2D_F32 || h->nclass > 3)
        return set_error(WAVE2D_ERR_ARG, "the streaming kernel needs an FP32 handle with four level planes");
    // class-chain handles: the stencil of their one to three classes
    const int points = h->nclass == 0 ? h->scheme : h->nclass == 1 ? 5 : h->nclass == 2 ? 9 : 13;
    switch (points) {
        case 5: return launch_stream_s<5>(h);
        case 9: return launch_stream_s<9>(h);
        default: return launch_stream_s<13>(h);
    }
}

}  // namespace w2d
