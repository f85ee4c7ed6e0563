// Kernel launchers for storage type __half (arithmetic in float).
#include "rpk_ops.cuh"

namespace rpk {
template struct Ops<__half, float>;
}  // namespace rpk
