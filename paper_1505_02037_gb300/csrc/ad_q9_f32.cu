// 37-field scheme: kernel instantiations for Q = 9, F32 storage.
#include "ad.cuh"

namespace lbnr {
namespace ad {
Table table_q9_f32() { return make_table<9, float>(); }
}  // namespace ad
}  // namespace lbnr
