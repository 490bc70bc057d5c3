"""Build the CUDA library ``libtmotif.so`` in-tree with nvcc for sm_103a."""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libtmotif.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC,-O2",
    "--expt-relaxed-constexpr",
]


# The kernel sources the library compiles again at run time for one tree
# (tm_codegen.cpp, NVRTC): embedded as text in the library.
KERNEL_FILES = ("tm_device.h", "tm_kernel.cuh")
KERNEL_INC = os.path.join(CSRC, "tm_kernel_src.inc")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def write_kernel_inc() -> None:
    """tm_kernel_src.inc: {name, text} of each kernel source, as raw strings."""
    parts = ["// generated by build.py from " + ", ".join(KERNEL_FILES) + "; do not edit",
             "struct KernelFile { const char *name; const char *text; };",
             "static const KernelFile kKernelFiles[] = {"]
    for name in KERNEL_FILES:
        text = open(os.path.join(CSRC, name)).read()
        assert ")TMSRC\"" not in text
        parts.append('    {"%s", R"TMSRC(%s)TMSRC"},' % (name, text))
    parts.append("};")
    body = "\n".join(parts) + "\n"
    if not os.path.exists(KERNEL_INC) or open(KERNEL_INC).read() != body:
        with open(KERNEL_INC + ".tmp", "w") as f:
            f.write(body)
        os.replace(KERNEL_INC + ".tmp", KERNEL_INC)


# Builds of the same sources with extra definitions, for tests only:
#   check: every data-dependent index of the mining kernel is checked (TM_ECHECK);
#   waits: a claimed task's payload wait is bounded at 16 polls and donors
#          pause ~0.2 ms before publishing, so that a test can make it run out.
VARIANTS = {
    None: [],
    "check": ["-DTM_CHECK=1"],
    "waits": ["-DTM_TEST_READY_SPINS=16", "-DTM_TEST_PUBLISH_PAUSE=200"],
}


def lib_path(variant=None) -> str:
    return LIB if variant is None else os.path.join(HERE, "libtmotif_%s.so" % variant)


def _deps():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in sources() + _deps())


def build(force: bool = False, verbose: bool = False, variant=None) -> str:
    """Compile every source to an object (in parallel), then link the library."""
    import concurrent.futures
    lib = lib_path(variant)
    if not force and not _stale(lib):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    write_kernel_inc()
    objdir = os.path.join(os.path.dirname(HERE), "_build", variant or "default")
    os.makedirs(objdir, exist_ok=True)
    deps_t = max(os.path.getmtime(p) for p in _deps())
    flags = NVCC_FLAGS + VARIANTS[variant] + ["-I" + INCLUDE] + (["-Xptxas=-v"] if verbose else [])

    def obj(src):
        o = os.path.join(objdir, os.path.basename(src) + ".o")
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(src), deps_t):
            cmd = [nvcc] + flags + ["-c", "-o", o + ".tmp", src]
            if verbose:
                print(" ".join(cmd))
            subprocess.check_call(cmd)
            os.replace(o + ".tmp", o)
        return o

    # the mining kernel's instantiations take minutes each: start them first
    order = sorted(sources(), key=lambda p: not os.path.basename(p).startswith("tm_kmine_"))
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(obj, order))
    tmp = lib + ".tmp%d" % os.getpid()
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(shutil.which(nvcc) or "/usr/local/cuda/bin/nvcc")),
                            "lib64")
    cmd = [nvcc] + NVCC_FLAGS + ["-shared", "-o", tmp] + objs + \
        ["-lcudart_static", "-lnvrtc", "-Xlinker", "-rpath=" + cuda_lib, "-lrt", "-ldl", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
