// 37-field scheme: kernel instantiations for Q = 19, F32 storage.
#include "ad.cuh"

namespace lbnr {
namespace ad {
Table table_q19_f32() { return make_table<19, float>(); }
}  // namespace ad
}  // namespace lbnr
