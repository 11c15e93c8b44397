// Kernel instantiations: D3Q19 velocity set, FP64 storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q19_s0() { return ops_for<19, 0>(); }
}  // namespace lbnr
