// Kernel instantiations: D3Q19 velocity set, BF16 deviation storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q19_s3() { return ops_for<19, 3>(); }
}  // namespace lbnr
