// Kernel instantiations: D1Q3 velocity set, FP64 storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q3_s0() { return ops_for<3, 0>(); }
}  // namespace lbnr
