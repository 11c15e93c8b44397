// Kernel instantiations: D2Q9 velocity set, FP32 storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q9_s1() { return ops_for<9, 1>(); }
}  // namespace lbnr
