// k_mine<true, true>: the extended schedules with work statistics.
#include "tm_instances.h"

namespace tmo {
template <> MineKernel mine_kernel<true, true>() { return dev::k_mine<true, true>; }
}  // namespace tmo
