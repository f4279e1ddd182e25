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

}  // namespace chain_detail
}  // namespace w2d
