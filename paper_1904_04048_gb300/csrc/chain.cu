// Launches of the derived-scheme kernels (kernels_chain.cuh) for a handle
// whose scheme is a prefix of nclass classes of the class chain: the first
// step and the one-node two-step (the TMA two-step is in chain_tma.cu).
#include "chain_launch.cuh"

namespace w2d {
using namespace chain_detail;

int chain_first_step(wave2d* h, const double* du0, const double* dv0, const ExactTab& ex, const Reduce& rd) {
    // u^0 -> plane 1 (u^{k-1}), u^1 -> plane 0; difference form: d^1 -> plane 2
    const Level L0 = h->level(h->diff_form ? 2 : 1), L1 = h->level(0);
    dispatch_dt(h->dtype, [&](auto DTc) {
        constexpr int DT = decltype(DTc)::value;
        dispatch_nc(h->nclass, [&](auto NCc) {
            constexpr int NC = decltype(NCc)::value;
            const CoefN<double, NC> ahalf = coef_n<double, NC>(h->ca, 0.5), b = coef_n<double, NC>(h->cb);
            dispatch_bool(h->bc == WAVE2D_BC_PERIODIC, [&](auto Pc) {
                dispatch_bool(h->tracking, [&](auto Tc) {
                    dispatch_bool(h->diff_form && DT == DT_F32, [&](auto Fc) {
                        constexpr bool F = decltype(Fc)::value && DT == DT_F32;
                        kc1_first_step<DT, NC, decltype(Pc)::value, decltype(Tc)::value, F>
                            <<<grid2d(h), dim3(32, 8), 0, h->stream>>>(du0, dv0, L0, L1, h->geo(), ahalf, b,
                                                                       h->tau, ex, rd, h->gw);
                    });
                });
            });
        });
    });
    W2D_LAUNCHED("derived-scheme first-step kernel launch");
    return WAVE2D_OK;
}

int chain_simple_step(wave2d* h, bool track, const ExactTab& ex, const Reduce& rd) {
    const Level cur = h->level(h->cur), nxt = h->level(h->prv);
    const Level dpl = h->diff_form ? h->level(2) : Level{nullptr, nullptr};
    dispatch_dt(h->dtype, [&](auto DTc) {
        constexpr int DT = decltype(DTc)::value;
        using V = typename St<DT>::V;
        dispatch_nc(h->nclass, [&](auto NCc) {
            constexpr int NC = decltype(NCc)::value;
            const CoefN<V, NC> a = coef_n<V, NC>(h->ca);
            dispatch_bool(h->bc == WAVE2D_BC_PERIODIC, [&](auto Pc) {
                dispatch_bool(track, [&](auto Tc) {
                    // difference sums exist for FP32 and FP64 storage, the
                    // difference form (which implies them) for FP32
                    const int mode = (h->diff_form && DT == DT_F32) ? 2 : (h->diff_sums && DT != DT_F32X2) ? 1 : 0;
                    auto go = [&](auto Dc, auto Fc) {
                        kc2_simple<DT, NC, decltype(Pc)::value, decltype(Tc)::value, decltype(Dc)::value,
                                   decltype(Fc)::value>
                            <<<grid2d(h), dim3(32, 8), 0, h->stream>>>(cur, nxt, h->geo(), a, ex, rd, h->gw, dpl);
                    };
                    if constexpr (DT == DT_F32) {
                        if (mode == 2) go(BC_<true>{}, BC_<true>{});
                        else if (mode == 1) go(BC_<true>{}, BC_<false>{});
                        else go(BC_<false>{}, BC_<false>{});
                    } else if constexpr (DT == DT_F64) {
                        if (mode == 1) go(BC_<true>{}, BC_<false>{});
                        else go(BC_<false>{}, BC_<false>{});
                    } else {
                        go(BC_<false>{}, BC_<false>{});
                    }
                });
            });
        });
    });
    W2D_LAUNCHED("derived-scheme two-step kernel launch");
    return WAVE2D_OK;
}

}  // namespace w2d
