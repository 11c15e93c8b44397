// 37-field scheme: kernel instantiations for Q = 19, F64 storage.
#include "ad.cuh"

namespace lbnr {
namespace ad {
Table table_q19_f64() { return make_table<19, double>(); }
}  // namespace ad
}  // namespace lbnr
