// k_mine<false, true>: counting launches that may use a thread tier, or
// sibling splitting and multi-offload.
#include "tm_instances.h"

namespace tmo {
template <> MineKernel mine_kernel<false, true>() { return dev::k_mine<false, true>; }
}  // namespace tmo
