// Instantiations of the derived-scheme launches for F64 storage.
#include "chain_launch.cuh"

namespace w2d {
namespace chain_detail {
template int chain_first_step_dt<DT_F64>(wave2d*, const double*, const double*, const ExactTab&, const Reduce&);
template int chain_simple_step_dt<DT_F64>(wave2d*, bool, const ExactTab&, const Reduce&);
}  // namespace chain_detail
}  // namespace w2d
