// Tree-specialised mining kernels: the code generation of Section 5.1
// ("GPU Code-generation") done by the runtime compiler.
//
// The paper generates, per motif group, a kernel whose nested loops follow
// the MG-Tree, so that the matching order, the mapped-vertex checks and the
// counters of each node are fixed in the code instead of looked up.  Here
// the mining kernel (tm_kernel.cuh) is compiled once per tree with NVRTC
// behind a generated prelude:
//   - the node, ref, window and query tables become __constant__ data of the
//     kernel (read through the constant cache, not from device memory);
//   - the tree's depth and vertex count size every per-level array and bound
//     every mapped-label loop (TM_K_MAXE, TM_K_MAXV), which sizes registers
//     and shared memory to the tree;
//   - the number of windows and counters, and whether any level scans the
//     global edge window, are compile-time constants.
// The generated program is compiled for sm_103a, loaded with
// cudaLibraryLoadData and kept in a process-wide cache keyed by its text, so
// trees of the same shape and windows share one compilation.
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <cstdio>
#include <cstdlib>

#include <chrono>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "tm_codegen.h"
#include "tm_internal.h"
#include "tm_kernel_src.inc"   // kKernelFiles: {name, text} of tm_device.h and tm_kernel.cuh (generated)

namespace tmo {
namespace {

std::mutex g_cache_mu;
std::map<std::string, std::unique_ptr<SpecKernel>> g_cache;   // by program text

// The prelude: limits, the tree's sizes and tables, then the kernel.
std::string program_text(const TreeImage &img, const HostTree &h) {
    const DevNode *nodes = (const DevNode *)img.bytes.data();
    const DevRef *refs = (const DevRef *)(img.bytes.data() + img.o_refs);
    const int64_t *deltas = (const int64_t *)(img.bytes.data() + img.o_deltas);
    const int8_t *qdmax = (const int8_t *)(img.bytes.data() + img.o_qdmax);
    int maxe = 1, maxv = 2;
    bool global = false;
    for (int i = 0; i < img.n_nodes; i++) {
        const DevNode &n = nodes[i];
        maxe = std::max(maxe, (int)n.k_end);
        for (int k = 0; k < n.k_end; k++) {
            maxv = std::max(maxv, 1 + std::max((int)n.eu[k], (int)n.ev[k]));
            if (k >= n.k_begin && k > 0 && n.eu[k] >= n.nvb[k] && n.ev[k] >= n.nvb[k]) global = true;
        }
    }
    (void)h;
    std::ostringstream o;
    o << "// generated: MG-Tree of " << img.n_nodes << " nodes, " << img.n_refs << " refs\n"
      << "#define TM_K_SPEC 1\n"
      << "#define TM_MAX_EDGES " << TM_MAX_EDGES << "\n#define TM_MAX_VERTICES " << TM_MAX_VERTICES << "\n"
      << "#define TM_MAX_DELTAS " << TM_MAX_DELTAS << "\n#define TM_WORK_FIELDS " << TM_WORK_FIELDS << "\n"
      << "#define TM_K_MAXE " << maxe << "\n#define TM_K_MAXV " << maxv << "\n"
      << "#define TM_K_NDELTAS " << img.n_deltas << "\n#define TM_K_NCOUNTERS " << img.n_counters << "\n"
      << "#define TM_K_NNODES " << img.n_nodes << "\n"
      << "#define TM_K_HAS_GLOBAL " << (global ? 1 : 0) << "\n"
      << "#include \"tm_device.h\"\n"
      << "namespace tmo {\nnamespace dev {\n";
    o << "__constant__ DevNode tmk_nodes[" << img.n_nodes << "] = {\n";
    for (int i = 0; i < img.n_nodes; i++) {
        const DevNode &n = nodes[i];
        o << "  {" << n.qmask << "ull, " << (int)n.k_begin << ", " << (int)n.k_end << ", " << (int)n.flags << ", "
          << (int)n.dmax << ", " << n.child_begin << ", " << (int)n.n_seq << ", " << (int)n.n_par << ", "
          << n.ref_begin << ", " << n.n_ref << ", " << n.parent << ", 0, {";
        for (int k = 0; k < maxe; k++) o << (k ? "," : "") << (int)n.eu[k];
        o << "}, {";
        for (int k = 0; k < maxe; k++) o << (k ? "," : "") << (int)n.ev[k];
        o << "}, {";
        for (int k = 0; k < maxe; k++) o << (k ? "," : "") << (int)n.nvb[k];
        o << "}},\n";
    }
    o << "};\n__constant__ DevRef tmk_refs[" << std::max(img.n_refs, 1) << "] = {";
    for (int i = 0; i < img.n_refs; i++)
        o << (i ? ", " : "") << "{" << refs[i].counter << ", " << refs[i].delta << ", " << refs[i].query << "}";
    if (img.n_refs == 0) o << "{0, 0, 0}";
    o << "};\n__constant__ int64_t tmk_deltas[" << std::max(img.n_deltas, 1) << "] = {";
    for (int i = 0; i < img.n_deltas; i++) o << (i ? ", " : "") << deltas[i] << "ll";
    if (img.n_deltas == 0) o << "0";
    o << "};\n__constant__ int8_t tmk_qdmax[64] = {";
    for (int q = 0; q < 64; q++) o << (q ? "," : "") << (int)qdmax[q];
    o << "};\n}  // namespace dev\n}  // namespace tmo\n#include \"tm_kernel.cuh\"\n";
    return o.str();
}

// FNV-1a of the whole program: the generated prelude and every embedded
// kernel source it includes (the on-disk cache must not outlive a kernel edit)
uint64_t fnv1a(const std::string &s) {
    uint64_t h = 1469598103934665603ull;
    auto add = [&h](const char *p, size_t n) {
        for (size_t i = 0; i < n; i++) h = (h ^ (unsigned char)p[i]) * 1099511628211ull;
    };
    add(s.data(), s.size());
    for (const auto &f : kKernelFiles) {
        add(f.name, strlen(f.name));
        add(f.text, strlen(f.text));
    }
    return h;
}

// On-disk cache of compiled programs, so that later processes skip the
// compilation: $TMOTIF_KERNEL_CACHE, else $XDG_CACHE_HOME/tmotif, else
// $HOME/.cache/tmotif; one file per program (the lowered kernel name, then
// the cubin), named by the program's hash and the runtime compiler's
// version.  Unwritable or absent directories only disable the cache.
std::string disk_path(uint64_t hash) {
    std::string dir;
    if (const char *d = getenv("TMOTIF_KERNEL_CACHE")) dir = d;
    else if (const char *x = getenv("XDG_CACHE_HOME")) dir = std::string(x) + "/tmotif";
    else if (const char *h = getenv("HOME")) dir = std::string(h) + "/.cache/tmotif";
    if (dir.empty()) return "";
    int major = 0, minor = 0;
    nvrtcVersion(&major, &minor);
    char name[96];
    snprintf(name, sizeof(name), "/k_mine_sm103a_nvrtc%d.%d_%016llx.bin", major, minor, (unsigned long long)hash);
    return dir + name;
}

void disk_store(uint64_t hash, const std::string &lowered, const std::vector<char> &cubin) {
    const std::string path = disk_path(hash);
    if (path.empty()) return;
    const std::string dir = path.substr(0, path.rfind('/'));
    // create the directory (one level below an existing parent is enough here)
    mkdir(dir.substr(0, dir.rfind('/')).c_str(), 0755);
    mkdir(dir.c_str(), 0755);
    const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return;
    const uint32_t ln = (uint32_t)lowered.size();
    bool ok = fwrite(&ln, 4, 1, f) == 1 && fwrite(lowered.data(), 1, ln, f) == ln &&
              fwrite(cubin.data(), 1, cubin.size(), f) == cubin.size();
    ok = (fclose(f) == 0) && ok;
    if (ok) rename(tmp.c_str(), path.c_str());
    else remove(tmp.c_str());
}

bool disk_load(uint64_t hash, std::string *lowered, std::vector<char> *cubin) {
    const std::string path = disk_path(hash);
    if (path.empty()) return false;
    FILE *f = fopen(path.c_str(), "rb");
    if (!f) return false;
    uint32_t ln = 0;
    bool ok = fread(&ln, 4, 1, f) == 1 && ln > 0 && ln < 4096;
    if (ok) {
        lowered->resize(ln);
        ok = fread(&(*lowered)[0], 1, ln, f) == ln;
    }
    if (ok) {
        char buf[1 << 16];
        size_t n;
        while ((n = fread(buf, 1, sizeof(buf), f)) > 0) cubin->insert(cubin->end(), buf, buf + n);
        ok = !cubin->empty();
    }
    fclose(f);
    return ok;
}

int load_cubin(const std::vector<char> &cubin, const std::string &lowered, SpecKernel *k);

// Compile one program; on success fills k (kernels loaded, not yet on a
// device).  With load == false only the compilation runs (no device needed).
int compile(const std::string &src, SpecKernel *k, bool load) {
    auto t0 = std::chrono::steady_clock::now();
    std::vector<const char *> names, texts;
    for (const auto &f : kKernelFiles) {
        names.push_back(f.name);
        texts.push_back(f.text);
    }
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "tm_spec.cu", (int)names.size(), texts.data(), names.data()) !=
        NVRTC_SUCCESS) {
        set_error("tm_tree_compile: nvrtcCreateProgram failed");
        return TM_ECUDA;
    }
    const char *expr = "tmo::dev::k_mine<false, false>";   // counting launches without a thread tier
    nvrtcAddNameExpression(prog, expr);
    // a compile-only check also asks the assembler for its register and spill report
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "-DNDEBUG",
                          "--ptxas-options=-v"};
    const int n_opts = (int)(sizeof(opts) / sizeof(opts[0])) - (load ? 1 : 0);
    nvrtcResult r = nvrtcCompileProgram(prog, n_opts, opts);
    size_t log_n = 0;
    nvrtcGetProgramLogSize(prog, &log_n);
    std::string log(log_n, '\0');
    if (log_n) nvrtcGetProgramLog(prog, &log[0]);
    if (r != NVRTC_SUCCESS) {
        set_error("tm_tree_compile: " + std::string(nvrtcGetErrorString(r)) + ": " + log.substr(0, 2000));
        nvrtcDestroyProgram(&prog);
        return TM_ECUDA;
    }
    if (!load) {                         // "Used N registers", "M bytes spill stores"
        const size_t u = log.find("Used ");
        if (u != std::string::npos) k->registers = atoi(log.c_str() + u + 5);
        const size_t sp = log.find(" bytes spill stores");
        if (sp != std::string::npos) {
            size_t b = log.rfind(' ', sp - 1);
            k->local_bytes = atoi(log.c_str() + (b == std::string::npos ? 0 : b + 1));
        }
        const size_t sm = log.find(" bytes smem");
        if (sm != std::string::npos) {
            size_t b = log.rfind(' ', sm - 1);
            k->static_smem = atoi(log.c_str() + (b == std::string::npos ? 0 : b + 1));
        }
    }
    const char *ln = nullptr;
    nvrtcGetLoweredName(prog, expr, &ln);
    const std::string lowered = ln ? ln : "";
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    std::vector<char> cubin(n);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    k->compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    disk_store(k->hash, lowered, cubin);   // a check compiles the same program: later loads reuse it
    if (!load) return TM_OK;
    return load_cubin(cubin, lowered, k);
}

// Load a compiled program and look up its kernel.
int load_cubin(const std::vector<char> &cubin, const std::string &lowered, SpecKernel *k) {
    cudaError_t e = cudaLibraryLoadData(&k->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) {
        set_error(std::string("tm_tree_compile: cudaLibraryLoadData: ") + cudaGetErrorString(e));
        return TM_ECUDA;
    }
    e = cudaLibraryGetKernel(&k->kern, k->lib, lowered.c_str());
    if (e != cudaSuccess) {
        set_error(std::string("tm_tree_compile: cudaLibraryGetKernel: ") + cudaGetErrorString(e));
        return TM_ECUDA;
    }
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, (const void *)k->kern) == cudaSuccess) {
        k->registers = fa.numRegs;
        k->local_bytes = (int)fa.localSizeBytes;
        k->static_smem = (int)fa.sharedSizeBytes;
    }
    return TM_OK;
}

// The kernel for one tree image, from the cache or compiled now.
int kernel_for(const TreeImage &img, const HostTree &h, bool load, const SpecKernel **out, bool *compiled) {
    const std::string src = program_text(img, h);
    if (!load) {                         // a check: compile, keep only the report
        SpecKernel *k = new SpecKernel();
        k->hash = fnv1a(src);
        int rc = compile(src, k, false);
        if (rc != TM_OK) {
            delete k;
            return rc;
        }
        *out = k;                        // released by the caller
        *compiled = true;
        return TM_OK;
    }
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_cache.find(src);
        if (it != g_cache.end()) {
            *out = it->second.get();
            *compiled = false;
            return TM_OK;
        }
    }
    std::unique_ptr<SpecKernel> k(new SpecKernel());
    k->hash = fnv1a(src);
    std::string lowered;
    std::vector<char> cubin;
    bool fresh = true;
    if (disk_load(k->hash, &lowered, &cubin) && load_cubin(cubin, lowered, k.get()) == TM_OK) {
        fresh = false;                   // compiled by an earlier process
    } else {
        k.reset(new SpecKernel());
        k->hash = fnv1a(src);
        TM_TRY(compile(src, k.get(), true));
    }
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto &slot = g_cache[src];
    if (!slot) slot = std::move(k);     // another thread may have compiled the same program meanwhile
    *out = slot.get();
    *compiled = fresh;
    return TM_OK;
}

}  // namespace

int tree_compile(tm_tree *tr, uint32_t flags, tm_compile_info *info) {
    if (tr->h.nodes.size() > (size_t)TM_SPEC_MAX_NODES) {
        set_error("tm_tree_compile: trees of more than TM_SPEC_MAX_NODES nodes are counted by the table-driven kernel");
        return TM_EUNSUPPORTED;
    }
    auto t0 = std::chrono::steady_clock::now();
    const bool chains = (flags & TM_COMPILE_CHAINS) != 0;
    const bool check = (flags & TM_COMPILE_CHECK) != 0;
    const int n_prog = 1 + (chains ? (int)tr->chains.size() : 0);
    std::vector<TreeImage> imgs(n_prog);
    imgs[0] = tr->image;
    for (int i = 1; i < n_prog; i++) tree_image(tr->chains[i - 1], true, &imgs[i]);
    std::vector<const SpecKernel *> ks(n_prog, nullptr);
    std::vector<int> rc(n_prog, TM_OK);
    std::vector<char> fresh(n_prog, 0);
    std::vector<std::string> err(n_prog);
    // independent programs compile on as many host threads
    const int n_thr = std::max(1, std::min(n_prog, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    std::mutex next_mu;
    int next = 0;
    for (int w = 0; w < n_thr; w++)
        pool.emplace_back([&]() {
            while (true) {
                int i;
                {
                    std::lock_guard<std::mutex> lk(next_mu);
                    if (next >= n_prog) return;
                    i = next++;
                }
                bool c = false;
                rc[i] = kernel_for(imgs[i], i == 0 ? tr->h : tr->chains[i - 1], !check, &ks[i], &c);
                fresh[i] = c;
                if (rc[i] != TM_OK) err[i] = tm_last_error();
            }
        });
    for (auto &t : pool) t.join();
    for (int i = 0; i < n_prog; i++)
        if (rc[i] != TM_OK) {
            if (check)                   // a check's records of the programs that did compile
                for (const SpecKernel *k : ks) delete k;
            set_error(err[i]);
            return rc[i];
        }
    if (!check) {
        std::lock_guard<std::mutex> lk(*(std::mutex *)tr->mutex);
        tr->spec_tree = ks[0];
        if (chains) tr->spec_chains.assign(ks.begin() + 1, ks.end());
    }
    std::unique_ptr<const SpecKernel> report(check ? ks[0] : nullptr);   // a check's own record
    if (check)
        for (int i = 1; i < n_prog; i++) delete ks[i];
    if (info) {
        memset(info, 0, sizeof(*info));
        info->kernels = n_prog;
        for (int i = 0; i < n_prog; i++) info->compiled += fresh[i];
        info->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ks[0]) {
            info->registers = ks[0]->registers;
            info->local_bytes = ks[0]->local_bytes;
            info->static_smem = ks[0]->static_smem;
            info->source_hash = ks[0]->hash;
        }
    }
    return TM_OK;
}

const SpecKernel *spec_kernel(const tm_tree *tr, int which) {
    std::lock_guard<std::mutex> lk(*(std::mutex *)tr->mutex);
    if (which == 0) return tr->spec_tree;
    if (which - 1 < (int)tr->spec_chains.size()) return tr->spec_chains[which - 1];
    return nullptr;
}

}  // namespace tmo
