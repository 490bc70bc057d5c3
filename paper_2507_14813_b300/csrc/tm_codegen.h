// Tree-specialised kernels (tm_codegen.cpp): compiled per MG-Tree at run time.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tmotif.h"

struct tm_tree;

namespace tmo {

// One compiled program: the mining kernel's counting launch specialised to
// one tree image.  Owned by the process-wide cache.
struct SpecKernel {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;                 // k_mine<false>
    int per_sm[64] = {0};                        // CTAs per SM by device (0: not yet computed)
    int registers = 0, local_bytes = 0, static_smem = 0;
    double compile_ms = 0;
    uint64_t hash = 0;                           // of the generated program text
};

// tm_tree_compile: the MG-Tree's kernel (and the chains' with TM_COMPILE_CHAINS)
int tree_compile(tm_tree *tr, uint32_t flags, tm_compile_info *info);
// the kernel compiled for tree `which` (0 = MG-Tree, 1 + i = chain i), or null
const SpecKernel *spec_kernel(const tm_tree *tr, int which);

}  // namespace tmo
