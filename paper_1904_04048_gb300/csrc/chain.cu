// Launches of the derived-scheme kernels (kernels_chain.cuh) for a handle
// whose scheme is a prefix of nclass classes of the class chain: the first
// step and the one-node two-step, dispatched to the per-storage-type
// instantiations (chain_f32.cu, chain_f64.cu, chain_f32x2.cu); the TMA
// two-step is in chain_tma.cu.
#include "chain_launch.cuh"

namespace w2d {
using namespace chain_detail;

int chain_first_step(wave2d* h, const double* du0, const double* dv0, const ExactTab& ex, const Reduce& rd) {
    switch (h->dtype) {
        case DT_F64: return chain_first_step_dt<DT_F64>(h, du0, dv0, ex, rd);
        case DT_F32: return chain_first_step_dt<DT_F32>(h, du0, dv0, ex, rd);
        default: return chain_first_step_dt<DT_F32X2>(h, du0, dv0, ex, rd);
    }
}

int chain_simple_step(wave2d* h, bool track, const ExactTab& ex, const Reduce& rd) {
    switch (h->dtype) {
        case DT_F64: return chain_simple_step_dt<DT_F64>(h, track, ex, rd);
        case DT_F32: return chain_simple_step_dt<DT_F32>(h, track, ex, rd);
        default: return chain_simple_step_dt<DT_F32X2>(h, track, ex, rd);
    }
}

}  // namespace w2d
