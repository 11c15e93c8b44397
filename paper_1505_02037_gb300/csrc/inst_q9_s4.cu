// Kernel instantiations: D2Q9 velocity set, FP16 deviation storage.
#include <cstdio>

#include "instantiate.cuh"

namespace lbnr {
const Ops* ops_q9_s4() { return ops_for<9, 4>(); }
}  // namespace lbnr
