// 37-field scheme: kernel instantiations for Q = 3, F64 storage.
#include "ad.cuh"

namespace lbnr {
namespace ad {
Table table_q3_f64() { return make_table<3, double>(); }
}  // namespace ad
}  // namespace lbnr
