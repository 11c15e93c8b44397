// Kernel instantiations: D2Q9 velocity set, FP64 storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q9_s0() { return ops_for<9, 0>(); }
}  // namespace lbnr
