// Kernel instantiations: D2Q9 velocity set, BF16 deviation storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q9_s3() { return ops_for<9, 3>(); }
}  // namespace lbnr
