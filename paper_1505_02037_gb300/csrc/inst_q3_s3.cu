// Kernel instantiations: D1Q3 velocity set, BF16 deviation storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q3_s3() { return ops_for<3, 3>(); }
}  // namespace lbnr
