// Kernel launchers for storage type float (arithmetic in float).
#include "rpk_ops.cuh"

namespace rpk {
template struct Ops<float, float>;
}  // namespace rpk
