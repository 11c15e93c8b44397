// Kernel instantiations: D1Q3 velocity set, FP32 storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q3_s1() { return ops_for<3, 1>(); }
}  // namespace lbnr
