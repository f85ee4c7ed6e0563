// Kernel launchers for storage type __nv_bfloat16 (arithmetic in float).
#include "rpk_ops.cuh"

namespace rpk {
template struct Ops<__nv_bfloat16, float>;
}  // namespace rpk
