// The table-driven mining kernel k_mine<kStats, kExt> (tm_kernel.cuh) as
// host launch handles.  Each instantiation is compiled in a translation unit
// of its own (tm_kmine_*.cu), so that the four build in parallel and no other
// source instantiates the kernel; the host code reaches them only through
// mine_kernel<kStats, kExt>().
#pragma once

#include "tm_kernel.cuh"

namespace tmo {

using MineKernel = void (*)(dev::Params);

template <bool kStats, bool kExt>
MineKernel mine_kernel();

template <> MineKernel mine_kernel<false, false>();   // counting (tm_kmine_count.cu)
template <> MineKernel mine_kernel<true, false>();    // counting with work statistics (tm_kmine_stats.cu)
template <> MineKernel mine_kernel<false, true>();    // with the extended schedules (tm_kmine_ext.cu)
template <> MineKernel mine_kernel<true, true>();     // both (tm_kmine_ext_stats.cu)

}  // namespace tmo
