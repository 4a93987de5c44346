// noalloc.cu -- petfmm_tree_noalloc: the quadtree build (binning, stable
// z-order sort, leaf ranges) for callers that must not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: a host application whose
// own caching allocator has already reserved the GPU's memory (a stray
// allocation can fail or fragment its pool), code with a fixed, audited
// device-memory budget, and latency-sensitive loops that cannot pay for
// cudaMalloc/cudaFree, which may synchronise the whole device.  For them this
// entry point keeps every intermediate buffer in one file-scope
// __device__ array of fixed size (PETFMM_NOALLOC_MAX_N particles' worth,
// about 16.3 MB), which every GPU that loads the library holds until the
// process exits.  The caller passes the inputs and the outputs.
//
// The array is one resource shared by every call: it keeps the previous
// call's contents, calls that overlap on the GPU (different streams, or
// different host threads) race on it, and each call clears the words that
// must start at zero.  Host code cannot use the array's name as a device
// address; its address is fetched with cudaGetSymbolAddress, with the device
// current, during the first call in each CUDA context (for the usual primary
// context: once per device), so that first call should come before any
// stream capture.  The cache is keyed by the context's unique ID, so a
// context made after cudaDeviceReset (or a non-primary context) gets its own
// lookup instead of a stale address.  The array itself is created when this
// file's device code is loaded onto the device: at the first lookup under
// lazy module loading (the CUDA default), else when the context is created;
// if the device has no room for it then, the call returns PETFMM_ENOMEM.
#include <cuda.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/petfmm.h"
#include "kernels.cuh"

using namespace petfmm;

namespace {

constexpr int64_t kMaxN = PETFMM_NOALLOC_MAX_N;
constexpr int64_t kRsBlocks = (kMaxN + 4095) / 4096;     // radix tiles of 4096 keys
// radix scratch: per-tile digit counts and the partial sums of their scan
// (fewer than 1024 words)
constexpr int64_t kSortWords = 256 * kRsBlocks + 1024;
constexpr int64_t kDescBytes = 4096;                     // InstDesc + Tasks
constexpr int64_t kScratchBytes = 4 * (4 * kMaxN + kSortWords + 16) + kDescBytes;

// The scratch: keys A, keys B, values A, values B (uint32 each), the radix
// sort's scratch, a status word, then the launch descriptors.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;

// Driver entry points for the current context and its unique ID, fetched
// through the runtime (no link-time dependency on the driver library).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

struct AddrEntry {
    unsigned long long ctx_id = 0;  // 0: unused slot
    void *addr = nullptr;
};
AddrEntry g_addr[64];  // per CUDA context: device address of g_noalloc_scratch
int g_next = 0;        // slot to overwrite when all 64 are taken

int map_lookup_error(cudaError_t e) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PETFMM_ENOMEM : PETFMM_ECUDA;
}

int scratch_address(void **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaError_t e = cudaSuccess;
    if (!g_ctx_current || !g_ctx_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                             &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            cudaGetLastError();
            return PETFMM_ECUDA;
        }
        g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS) return PETFMM_ECUDA;
    if (!ctx) {
        // no context on this thread yet: the runtime's first call makes the
        // current device's primary context current
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return map_lookup_error(e);
        if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return PETFMM_ECUDA;
    }
    unsigned long long id = 0;
    if (g_ctx_id(ctx, &id) != CUDA_SUCCESS || id == 0) return PETFMM_ECUDA;
    for (const AddrEntry &a : g_addr)
        if (a.ctx_id == id) {
            *out = a.addr;
            return PETFMM_OK;
        }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return map_lookup_error(e);
    if (!p) return PETFMM_ECUDA;
    AddrEntry *slot = nullptr;
    for (AddrEntry &a : g_addr)
        if (a.ctx_id == 0) {
            slot = &a;
            break;
        }
    if (!slot) {
        slot = &g_addr[g_next];
        g_next = (g_next + 1) % 64;
    }
    slot->ctx_id = id;
    slot->addr = p;
    *out = p;
    return PETFMM_OK;
}

}  // namespace

extern "C" int petfmm_tree_noalloc(const petfmm_domain *dom, int levels, int dtype, int64_t n,
                                   const void *x, const void *y, uint32_t *keys, uint32_t *perm,
                                   uint32_t *start, void *cuda_stream) {
    if (!dom || !(dom->width > 0.0) || levels < 1 || levels > MAX_L || n < 0 || !perm || !start)
        return PETFMM_EINVAL;
    if (dtype != PETFMM_F64 && dtype != PETFMM_F32) return PETFMM_EINVAL;
    if (n > 0 && (!x || !y)) return PETFMM_EINVAL;
    if (n > kMaxN) return PETFMM_ENOMEM;  // the fixed scratch holds at most kMaxN particles
    if (radix_blocks(n) > kRsBlocks || radix_scratch_words(n) > kSortWords) return PETFMM_ENOMEM;
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned char *b = static_cast<unsigned char *>(base);
    uint32_t *kA = reinterpret_cast<uint32_t *>(b);
    uint32_t *kB = kA + kMaxN;
    uint32_t *vA = kB + kMaxN;
    uint32_t *vB = vA + kMaxN;
    uint32_t *sortw = vB + kMaxN;
    int *status = reinterpret_cast<int *>(sortw + kSortWords);
    unsigned char *descs = reinterpret_cast<unsigned char *>(status + 16);

    // launch descriptors of this call: one instance, one task per stage
    struct {
        InstDesc d;
        Task t[3];  // binning (particles), leaf starts (4^L + 1), unused
    } h;
    std::memset(&h, 0, sizeof(h));
    inst_set_domain(h.d, dom->x0, dom->y0, dom->width, levels);
    h.d.L = levels;
    h.d.n = n;
    h.d.x = x;
    h.d.y = y;
    h.t[0] = Task{0, levels, n, 0};
    h.t[1] = Task{0, levels, (int64_t(1) << (2 * levels)) + 1, 0};
    static_assert(sizeof(h) <= kDescBytes, "descriptor space");
    InstDesc *dd = reinterpret_cast<InstDesc *>(descs);
    Task *dt = reinterpret_cast<Task *>(descs + sizeof(InstDesc));
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return PETFMM_ECUDA;
    if (cudaMemcpyAsync(dd, &h, sizeof(h), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return PETFMM_ECUDA;
    uint64_t launches = 0;
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        e = launch_morton(dt, 1, (n + 255) / 256, dd, dtype == PETFMM_F32, kA, nullptr, status, st,
                          &launches);
        if (e == cudaSuccess && keys) e = cudaMemcpyAsync(keys, kA, size_t(n) * 4, cudaMemcpyDeviceToDevice, st);
        bool in_first = true;
        if (e == cudaSuccess) e = radix_sort(kA, vA, kB, vB, n, 2 * levels, sortw, &in_first, st, &launches);
        const uint32_t *sk = in_first ? kA : kB;
        const uint32_t *sv = in_first ? vA : vB;
        if (e == cudaSuccess) e = cudaMemcpyAsync(perm, sv, size_t(n) * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = launch_leaf_start(dt + 1, 1, ((int64_t(1) << (2 * levels)) + 1 + 255) / 256, dd, sk, start, st,
                                  &launches);
    } else {
        e = cudaMemsetAsync(start, 0, ((size_t(1) << (2 * levels)) + 1) * 4, st);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PETFMM_ECUDA;
    }
    int hs = 0;
    if (cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return PETFMM_ECUDA;
    }
    return hs;
}
