// Host-side helpers shared by the launch files of the derived-scheme
// kernels (chain.cu, chain_tma.cu).
#pragma once
#include <algorithm>
#include <type_traits>

#include "kernels_chain.cuh"
#include "wave2d_impl.cuh"

namespace w2d {
namespace chain_detail {

template <int V>
using IC = std::integral_constant<int, V>;
template <bool V>
using BC_ = std::integral_constant<bool, V>;

template <typename Fn>
inline void dispatch_nc(int nc, Fn&& fn) {
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
inline void dispatch_dt(int dt, Fn&& fn) {
    switch (dt) {
        case DT_F64: fn(IC<DT_F64>{}); break;
        case DT_F32: fn(IC<DT_F32>{}); break;
        default: fn(IC<DT_F32X2>{}); break;
    }
}
template <typename Fn>
inline void dispatch_bool(bool v, Fn&& fn) {
    if (v) fn(BC_<true>{});
    else fn(BC_<false>{});
}

inline df split(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
template <typename V, int NC>
inline CoefN<V, NC> coef_n(const double* c, double scale = 1.0) {
    CoefN<V, NC> r;
    for (int q = 0; q < NC; ++q) {
        const double v = c[q] * scale;
        if constexpr (std::is_same<V, df>::value) r.a[q] = split(v);
        else r.a[q] = (V)v;
    }
    return r;
}

inline dim3 grid2d(const wave2d* h) { return dim3((h->nx + 31) / 32, (h->ny + 7) / 8); }

template <typename Fn>
inline void dispatch_bcm(int bc, Fn&& fn) {
    switch (bc) {
        case WAVE2D_BC_PERIODIC: fn(IC<BCM_PERIODIC>{}); break;
        case WAVE2D_BC_ODD: fn(IC<BCM_ODD>{}); break;
        default: fn(IC<BCM_ZERO>{}); break;
    }
}

// First step and one-node two-step of a derived-scheme handle whose storage
// type is DT (instantiated once per type, in chain_f32.cu, chain_f64.cu and
// chain_f32x2.cu, so the three compile in parallel).
template <int DT>
int chain_first_step_dt(wave2d* h, const double* du0, const double* dv0, const ExactTab& ex, const Reduce& rd) {
    // u^0 -> plane 1 (u^{k-1}), u^1 -> plane 0; difference form: d^1 -> plane dpl
    const Level L0 = h->level(h->diff_form ? h->dpl : 1), L1 = h->level(0);
    dispatch_nc(h->nclass, [&](auto NCc) {
        constexpr int NC = decltype(NCc)::value;
        const CoefN<double, NC> ahalf = coef_n<double, NC>(h->ca, 0.5), b = coef_n<double, NC>(h->cb);
        dispatch_bcm(h->bc, [&](auto Bc) {
            dispatch_bool(h->tracking, [&](auto Tc) {
                dispatch_bool(h->diff_form && DT == DT_F32, [&](auto Fc) {
                    constexpr bool F = decltype(Fc)::value && DT == DT_F32;
                    kc1_first_step<DT, NC, decltype(Bc)::value, decltype(Tc)::value, F>
                        <<<grid2d(h), dim3(32, 8), 0, h->stream>>>(du0, dv0, L0, L1, h->geo(), ahalf, b, h->tau, ex,
                                                                   rd, h->gw);
                });
            });
        });
    });
    W2D_LAUNCHED("derived-scheme first-step kernel launch");
    return WAVE2D_OK;
}

template <int DT>
int chain_simple_step_dt(wave2d* h, bool track, const ExactTab& ex, const Reduce& rd) {
    using V = typename St<DT>::V;
    const Level cur = h->level(h->cur), nxt = h->level(h->prv);
    const Level dpl = h->diff_form ? h->level(h->dpl) : Level{nullptr, nullptr};
    // difference sums exist for FP32 and FP64 storage, the difference form
    // (which implies them) for FP32
    const int mode = (h->diff_form && DT == DT_F32) ? 2 : (h->diff_sums && DT != DT_F32X2) ? 1 : 0;
    dispatch_nc(h->nclass, [&](auto NCc) {
        constexpr int NC = decltype(NCc)::value;
        const CoefN<V, NC> a = coef_n<V, NC>(h->ca);
        dispatch_bcm(h->bc, [&](auto Bc) {
            dispatch_bool(track, [&](auto Tc) {
                auto go = [&](auto Dc, auto Fc) {
                    kc2_simple<DT, NC, decltype(Bc)::value, decltype(Tc)::value, decltype(Dc)::value,
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
    W2D_LAUNCHED("derived-scheme two-step kernel launch");
    return WAVE2D_OK;
}

extern template int chain_first_step_dt<DT_F64>(wave2d*, const double*, const double*, const ExactTab&,
                                                const Reduce&);
extern template int chain_first_step_dt<DT_F32>(wave2d*, const double*, const double*, const ExactTab&,
                                                const Reduce&);
extern template int chain_first_step_dt<DT_F32X2>(wave2d*, const double*, const double*, const ExactTab&,
                                                  const Reduce&);
extern template int chain_simple_step_dt<DT_F64>(wave2d*, bool, const ExactTab&, const Reduce&);
extern template int chain_simple_step_dt<DT_F32>(wave2d*, bool, const ExactTab&, const Reduce&);
extern template int chain_simple_step_dt<DT_F32X2>(wave2d*, bool, const ExactTab&, const Reduce&);

}  // namespace chain_detail
}  // namespace w2d
