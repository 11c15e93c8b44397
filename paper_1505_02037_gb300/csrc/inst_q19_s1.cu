// Kernel instantiations: D3Q19 velocity set, FP32 storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q19_s1() { return ops_for<19, 1>(); }
}  // namespace lbnr
