// Kernel instantiations: D3Q19 velocity set, FP16 deviation storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q19_s4() { return ops_for<19, 4>(); }
}  // namespace lbnr
