// k_mine<false, false>: the counting launches.
#include "tm_instances.h"

namespace tmo {
template <> MineKernel mine_kernel<false, false>() { return dev::k_mine<false, false>; }
}  // namespace tmo
