// Kernel instantiations: D2Q9 velocity set, FP32 deviation storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q9_s2() { return ops_for<9, 2>(); }
}  // namespace lbnr
