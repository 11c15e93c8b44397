// Kernel instantiations: D1Q3 velocity set, FP32 deviation storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q3_s2() { return ops_for<3, 2>(); }
}  // namespace lbnr
