// Kernel instantiations: D3Q19 velocity set, FP32 deviation storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q19_s2() { return ops_for<19, 2>(); }
}  // namespace lbnr
