// k_mine<true, false>: counting launches that also gather work statistics
// (tm_run_stats, per-root work).
#include "tm_instances.h"

namespace tmo {
template <> MineKernel mine_kernel<true, false>() { return dev::k_mine<true, false>; }
}  // namespace tmo
