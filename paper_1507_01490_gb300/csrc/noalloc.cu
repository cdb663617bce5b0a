// bcm_farness_all_noalloc: f(v) and r(v) of every vertex without allocating
// any memory.
//
// Some callers cannot allocate device memory at the moment they need this:
// a host framework may own all device memory through its own allocator, a
// latency-critical service may forbid allocation on its request path (a
// cudaMalloc can synchronise the device and stall other streams), and code
// that runs with a fixed memory budget cannot grow it on demand.  This entry
// point serves them: all of its working memory is one fixed array compiled
// into the library, and it calls no allocating routine.
//
// The array is shared by every call in the process on a given device and
// keeps the last call's contents; each call clears the parts that must start
// at zero.  Two calls whose work overlaps on the GPU (different streams, or
// different host threads on one device) use the same array at the same time
// and corrupt each other's results: order such calls on one stream or
// serialise them.
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "bcm.h"
#include "internal.h"

namespace bcm {

// 64 MiB: the CSR offsets narrowed to 32 bits, a source order, and the
// per-CTA wave slots (44 bytes per vertex each) for as many CTAs as fit.
constexpr size_t kNoAllocBytes = 64ull << 20;
constexpr uint32_t kNoAllocMaxN = 1250000;   // at least one CTA slot (44 bytes per vertex) fits

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocHeader {
    uint32_t head;
    int err;
    int csr_err;
    uint32_t pad;
    unsigned long long stats[ST_COUNT];
};

// Layout: header (256 bytes) | offsets u32[n+1] | order u32[n] | CTA slots.
constexpr size_t kHeaderBytes = 256;
static_assert(sizeof(NoAllocHeader) <= kHeaderBytes, "the header must fit before the offsets");
constexpr size_t noalloc_fixed_bytes(uint32_t n) {
    return kHeaderBytes + al256(((size_t)n + 1) * 4) + al256((size_t)n * 4);
}
static_assert(noalloc_fixed_bytes(kNoAllocMaxN) + slot_bytes(kNoAllocMaxN, 1) <= kNoAllocBytes,
              "at the vertex limit one CTA slot must still fit in the array");

__global__ void k_noalloc_identity(uint32_t* order, uint32_t n) {
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += stride) order[v] = (uint32_t)v;
}

// Device address of the array, looked up once per device (with that device
// current) on the first call there and kept for the life of the process.
// It belongs to the device's primary context (the one the runtime API uses);
// a cudaDeviceReset or a call made under another context would leave it
// stale, which is why both are outside what this entry point supports.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

static cudaError_t noalloc_base(int dev, void** out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace bcm

using namespace bcm;

// the message bcm_last_error() reports for this thread
static bcm_status noalloc_fail(bcm_status st, const char* msg) {
    set_error_message(msg);
    return st;
}

extern "C" bcm_status bcm_farness_all_noalloc(const uint64_t* row_ptr, const uint32_t* col, uint32_t n, uint64_t m,
                                              void* stream, uint64_t* farness, uint32_t* reach) {
    set_error_message("");
    if (!row_ptr || (m > 0 && !col) || !farness || !reach)
        return noalloc_fail(BCM_ERR_INVALID, "bcm_farness_all_noalloc: a pointer argument is NULL");
    if (n > kNoAllocMaxN) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "bcm_farness_all_noalloc: n = %u exceeds this variant's limit of %u vertices "
                 "(its fixed 64 MiB working array); use bcm_farness_all",
                 n, kNoAllocMaxN);
        return noalloc_fail(BCM_ERR_UNSUPPORTED, buf);
    }
    if (m >= (1ull << 32)) return noalloc_fail(BCM_ERR_UNSUPPORTED, "bcm_farness_all_noalloc: m must be below 2^32");
    if (n == 0) return BCM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_fail(BCM_ERR_CUDA, "cudaGetDevice failed");
    void* base = nullptr;
    cudaError_t e = noalloc_base(dev, &base);
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof(buf), "cudaGetSymbolAddress of the working array failed: %s", cudaGetErrorString(e));
        return noalloc_fail(BCM_ERR_CUDA, buf);
    }
    // layout: header | 32-bit offsets | source order | CTA slots
    char* p = (char*)base;
    NoAllocHeader* hdr = (NoAllocHeader*)p;
    uint32_t* rp32 = (uint32_t*)(p + kHeaderBytes);
    uint32_t* order = (uint32_t*)((char*)rp32 + al256(((size_t)n + 1) * 4));
    char* slots = (char*)order + al256((size_t)n * 4);
    const size_t fixed = noalloc_fixed_bytes(n);
    const size_t sb = slot_bytes(n, 1);
    const int per = cta_blocks_per_sm(1, 512);
    if (per <= 0) {
        const cudaError_t oe = cudaGetLastError();
        char buf[256];
        snprintf(buf, sizeof(buf), "bcm_farness_all_noalloc: the occupancy query of the wave kernel failed: %s",
                 cudaGetErrorString(oe));
        return noalloc_fail(BCM_ERR_CUDA, buf);
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0) {
        char buf[256];
        snprintf(buf, sizeof(buf), "bcm_farness_all_noalloc: reading the SM count failed: %s", cudaGetErrorString(e));
        return noalloc_fail(BCM_ERR_CUDA, buf);
    }
    size_t fit = (kNoAllocBytes - fixed) / sb;
    size_t blocks = (size_t)per * (size_t)sms;
    if (blocks > fit) blocks = fit;
    if (blocks < 1) return noalloc_fail(BCM_ERR_UNSUPPORTED, "bcm_farness_all_noalloc: graph too large for the array");

    // what must start at zero: the header and the slots this call uses
    if (cudaMemsetAsync(hdr, 0, sizeof(NoAllocHeader), s) != cudaSuccess ||
        cudaMemsetAsync(slots, 0, blocks * sb, s) != cudaSuccess)
        return noalloc_fail(BCM_ERR_CUDA, "clearing the working array failed");
    if (launch_validate(row_ptr, col, n, m, &hdr->csr_err, s) || launch_narrow_offsets(row_ptr, rp32, n, s))
        return noalloc_fail(BCM_ERR_CUDA, "CSR check kernels failed to launch");
    k_noalloc_identity<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0, s>>>(order, n);
    note_launch();

    WaveParams w;
    memset(&w, 0, sizeof(w));
    w.g.n = n;
    w.g.m = m;
    w.g.rp = rp32;
    w.g.col = col;
    w.g.order = order;
    w.sources = order;
    w.g.xlo = order;          // bounds are not read when nothing is cut
    w.g.xhi = order;
    w.g.rrp = rp32;
    w.g.rcol = col;
    w.exhaustive = 1;
    w.head = &hdr->head;
    w.n_end = n;
    w.out_far = (unsigned long long*)farness;
    w.out_reach = reach;
    w.slot_base = slots;
    w.slot_stride = sb;
    w.cta_entries = n;        // dense per-CTA slots (no hashed table: exhaustive runs never defer)
    w.stats = hdr->stats;
    w.err = &hdr->err;
    w.lock_limit_ns = 20ull * 1000 * 1000 * 1000;
    w.barrier_limit_ns = w.lock_limit_ns;
    int herr[2] = {0, 0};
    // a malformed CSR must not reach the wave kernel
    if (cudaMemcpyAsync(&herr[1], &hdr->csr_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return noalloc_fail(BCM_ERR_CUDA, "CSR check failed");
    if (herr[1]) return noalloc_fail(BCM_ERR_INVALID, "malformed CSR: row_ptr must rise from 0 to m and every col < n");
    if (launch_cta_waves(w, 1, (int)blocks, 512, s)) return noalloc_fail(BCM_ERR_CUDA, "wave kernel launch failed");
    if (cudaMemcpyAsync(&herr[0], &hdr->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return noalloc_fail(BCM_ERR_CUDA, "wave kernel failed");
    if (herr[0]) return noalloc_fail(BCM_ERR_TIMEOUT, "an in-kernel wait ran past its limit");
    return BCM_OK;
}
