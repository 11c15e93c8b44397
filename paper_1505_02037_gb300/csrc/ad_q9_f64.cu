// 37-field scheme: kernel instantiations for Q = 9, F64 storage.
#include "ad.cuh"

namespace lbnr {
namespace ad {
Table table_q9_f64() { return make_table<9, double>(); }
}  // namespace ad
}  // namespace lbnr
