// Kernel instantiations: D1Q3 velocity set, FP16 deviation storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q3_s4() { return ops_for<3, 4>(); }
}  // namespace lbnr
