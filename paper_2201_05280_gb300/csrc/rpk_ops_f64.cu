// Kernel launchers for storage type double (arithmetic in double).
#include "rpk_ops.cuh"

namespace rpk {
template struct Ops<double, double>;
}  // namespace rpk
