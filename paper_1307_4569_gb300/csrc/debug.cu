// Guard-zone bounds checking of the DGT_DEBUG build (see debug.h), and its C ABI.
#include "debug.h"

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "dgt.h"

namespace dgt {

#ifdef DGT_DEBUG

struct Zone {
    unsigned long long addr, bytes;
};
struct DbgErr {
    unsigned long long count;   // overwritten guard words since the last status read
    unsigned long long seq;     // check (launch) sequence number of the first of them
    unsigned long long addr;    // its zone
    unsigned long long word;    // its word index in the zone
};
struct HostZone {
    unsigned long long addr, bytes;
    const void* owner;          // the allocation it guards (persistent zones), else null
    unsigned long long tag;     // the call scope that registered it (transient zones), else 0
};

// every registered zone, one block per zone (grid-stride); a damaged word is re-armed so that
// each violation is counted once, and the first one since the last read is recorded
__global__ void guard_check_kernel(const Zone* __restrict__ z, int nz, DbgErr* err, unsigned long long seq) {
    for (int i = blockIdx.x; i < nz; i += gridDim.x) {
        unsigned int* p = reinterpret_cast<unsigned int*>(z[i].addr);
        const unsigned long long nw = z[i].bytes / 4;
        for (unsigned long long w = threadIdx.x; w < nw; w += blockDim.x) {
            if (p[w] != 0xFFFFFFFFu) {
                p[w] = 0xFFFFFFFFu;
                if (atomicAdd(&err->count, 1ull) == 0ull) {
                    err->seq = seq;
                    err->addr = z[i].addr;
                    err->word = w;
                }
            }
        }
    }
}

static std::recursive_mutex g_mu;
static std::vector<HostZone> g_zones;
static Zone* g_dz = nullptr;            // device snapshot of g_zones
static int g_dn = 0;
static bool g_dirty = false;
static DbgErr* g_derr = nullptr;        // device record
constexpr int kRing = 1 << 16;
static const char* g_names[kRing];      // check sequence number -> launch name
static unsigned long long g_seq = 0;
static unsigned long long g_tag = 0;

static size_t round4(size_t n) { return (n + 3) & ~(size_t)3; }

static cudaError_t ensure_record() {
    if (g_derr) return cudaSuccess;
    cudaError_t e = cudaMalloc(&g_derr, sizeof(DbgErr));
    if (e != cudaSuccess) return e;
    return cudaMemset(g_derr, 0, sizeof(DbgErr));
}

// replace the device snapshot after the zones changed; nothing that reads the old one is in
// flight after the synchronisation
static cudaError_t upload() {
    if (!g_dirty) return cudaSuccess;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    if (g_dz) cudaFree(g_dz);
    g_dz = nullptr;
    g_dn = 0;
    if (!g_zones.empty()) {
        std::vector<Zone> h(g_zones.size());
        for (size_t i = 0; i < h.size(); ++i) h[i] = {g_zones[i].addr, g_zones[i].bytes};
        e = cudaMalloc(&g_dz, sizeof(Zone) * h.size());
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(g_dz, h.data(), sizeof(Zone) * h.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        g_dn = (int)h.size();
    }
    g_dirty = false;
    return cudaSuccess;
}

cudaError_t dbg_malloc(void** p, size_t bytes) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    const size_t body = round4(bytes);
    char* base = nullptr;
    cudaError_t e = cudaMalloc(&base, kGuard + body + kGuard);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemset(base, 0xFF, kGuard)) != cudaSuccess ||
        (e = cudaMemset(base + kGuard + body, 0xFF, kGuard)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
        cudaFree(base);
        return e;
    }
    *p = base + kGuard;
    g_zones.push_back({(unsigned long long)base, kGuard, *p, 0});
    g_zones.push_back({(unsigned long long)(base + kGuard + body), kGuard, *p, 0});
    g_dirty = true;
    return cudaSuccess;
}

void dbg_free(void* p) {
    if (!p) return;
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    cudaDeviceSynchronize();
    g_zones.erase(std::remove_if(g_zones.begin(), g_zones.end(), [&](const HostZone& z) { return z.owner == p; }),
                  g_zones.end());
    g_dirty = true;
    upload();
    cudaFree(static_cast<char*>(p) - kGuard);
}

void dbg_after_launch(const char* name, cudaStream_t st) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (g_zones.empty() || upload() != cudaSuccess || ensure_record() != cudaSuccess) return;
    const unsigned long long seq = ++g_seq;
    g_names[seq % kRing] = name;
    guard_check_kernel<<<std::min(g_dn, 1024), 256, 0, st>>>(g_dz, g_dn, g_derr, seq);
    cudaGetLastError();
}

DbgScope::DbgScope(cudaStream_t st, char* base, const size_t* offsets, int n) {
    g_mu.lock();
    tag_ = ++g_tag;
    for (int i = 0; i < n; ++i) cudaMemsetAsync(base + offsets[i], 0xFF, kGuard, st);
    cudaStreamSynchronize(st);
    for (int i = 0; i < n; ++i) g_zones.push_back({(unsigned long long)(base + offsets[i]), kGuard, nullptr, tag_});
    if (n > 0) g_dirty = true;
}

DbgScope::~DbgScope() {
    cudaDeviceSynchronize();
    const unsigned long long t = tag_;
    const size_t before = g_zones.size();
    g_zones.erase(std::remove_if(g_zones.begin(), g_zones.end(), [&](const HostZone& z) { return z.tag == t; }),
                  g_zones.end());
    if (g_zones.size() != before) g_dirty = true;
    g_mu.unlock();
}

static int debug_status(unsigned long long* violations, long long* zone_offset, char* kernel, size_t kernel_len) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (violations) *violations = 0;
    if (zone_offset) *zone_offset = -1;
    if (kernel && kernel_len) kernel[0] = 0;
    if (cudaDeviceSynchronize() != cudaSuccess || ensure_record() != cudaSuccess) return DGT_ERR_CUDA;
    DbgErr h{};
    if (cudaMemcpy(&h, g_derr, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return DGT_ERR_CUDA;
    if (cudaMemset(g_derr, 0, sizeof(DbgErr)) != cudaSuccess) return DGT_ERR_CUDA;
    if (violations) *violations = h.count;
    if (h.count) {
        if (zone_offset) *zone_offset = (long long)(4 * h.word);
        const char* nm = h.seq + kRing > g_seq ? g_names[h.seq % kRing] : nullptr;
        if (kernel && kernel_len && nm) {
            std::strncpy(kernel, nm, kernel_len - 1);
            kernel[kernel_len - 1] = 0;
        }
    }
    return DGT_OK;
}

static int debug_touch(void* p) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (cudaMemset(p, 0, 4) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return DGT_ERR_CUDA;
    return DGT_OK;
}

#else

cudaError_t dbg_malloc(void** p, size_t bytes) { return cudaMalloc(p, bytes); }
void dbg_free(void* p) {
    if (p) cudaFree(p);
}
void dbg_after_launch(const char*, cudaStream_t) {}
DbgScope::DbgScope(cudaStream_t, char*, const size_t*, int) {}
DbgScope::~DbgScope() {}

#endif

// the first word of the trailing guard zone of an allocation of `bytes` bytes at p
int dbg_touch_trailing_guard(void* p, size_t bytes) {
#ifdef DGT_DEBUG
    return debug_touch(static_cast<char*>(p) + round4(bytes));
#else
    (void)p;
    (void)bytes;
    return DGT_ERR_UNSUPPORTED;
#endif
}

}  // namespace dgt

extern "C" int dgt_debug_build(void) { return dgt::kDebug ? 1 : 0; }

extern "C" int dgt_debug_status(unsigned long long* violations, long long* zone_offset, char* kernel,
                                size_t kernel_len) {
#ifdef DGT_DEBUG
    return dgt::debug_status(violations, zone_offset, kernel, kernel_len);
#else
    if (violations) *violations = 0;
    if (zone_offset) *zone_offset = -1;
    if (kernel && kernel_len) kernel[0] = 0;
    return DGT_ERR_UNSUPPORTED;
#endif
}
