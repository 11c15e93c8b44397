// 37-field scheme: kernel instantiations for Q = 3, F32 storage.
#include "ad.cuh"

namespace lbnr {
namespace ad {
Table table_q3_f32() { return make_table<3, float>(); }
}  // namespace ad
}  // namespace lbnr
