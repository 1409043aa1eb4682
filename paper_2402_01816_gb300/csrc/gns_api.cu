// gns_api.cu -- the C ABI: argument checks, status word, allocator hook,
// instrumentation.  Every sorting step runs in the library's own kernels.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "gns_device.cuh"
#include "gns_internal.h"

namespace gns {

std::atomic<uint64_t> g_launches{0};

// ---------------------------------------------------------------- status word
__device__ int g_status_word;   // per device: first device-side error since last read

namespace {
std::mutex g_status_mu;
std::vector<int*> g_status_ptrs;   // indexed by device ordinal
}

int* status_word_ptr()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mu);
    if ((int)g_status_ptrs.size() <= dev) g_status_ptrs.resize(dev + 1, nullptr);
    if (!g_status_ptrs[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
        g_status_ptrs[dev] = (int*)p;
    }
    return g_status_ptrs[dev];
}

int finish_call(int rc, cudaStream_t s)
{
    if (rc != GNS_OK) return rc;
    static const bool sync_status = [] {
        const char* e = getenv("GNS_SYNC_STATUS");
        return e && e[0] == '1';
    }();
    if (!sync_status) return rc;
    return gns_stream_status((gns_stream_t)s);
}

// ------------------------------------------------------------ allocator hook
namespace {
gns_alloc_fn g_alloc = nullptr;
gns_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;
}

// The default allocator is a dedicated stream-ordered memory pool per device
// whose release threshold is "never": freed workspace stays mapped for the next
// call instead of being unmapped at every synchronisation.
namespace {
std::mutex g_pool_mu;
std::vector<cudaMemPool_t> g_pools;   // indexed by device ordinal
}

cudaMemPool_t workspace_pool(int dev)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if ((int)g_pools.size() <= dev) g_pools.resize(dev + 1, nullptr);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}

void* ws_alloc(size_t bytes, cudaStream_t s)
{
    if (bytes == 0) bytes = 256;
    if (g_alloc) return g_alloc(bytes, (gns_stream_t)s, g_alloc_ctx);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaMemPool_t pool = workspace_pool(dev);
    if (!pool) return nullptr;
    void* p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void ws_free(void* p, cudaStream_t s)
{
    if (!p) return;
    if (g_free) {
        g_free(p, (gns_stream_t)s, g_alloc_ctx);
        return;
    }
    cudaFreeAsync(p, s);
}

// ------------------------------------------------------------ bounded waits
namespace {
std::atomic<uint64_t> g_wait_limit_ns{2000000000ull};
std::atomic<int64_t> g_debug_skip{-1};
}

uint64_t wait_limit_ns() { return g_wait_limit_ns.load(); }
int64_t take_debug_skip_publish() { return g_debug_skip.exchange(-1); }
std::atomic<uint32_t> g_debug_jitter{0};
uint32_t debug_jitter_ns() { return g_debug_jitter.load(); }

// ------------------------------------------------------------ profiling
namespace {
struct ProfRec {
    int kid;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_event_pool;
thread_local int g_pending_kid = -1;
thread_local cudaEvent_t g_pending_a = nullptr;
thread_local bool g_capturing = false;
thread_local uint64_t g_captured = 0;

cudaEvent_t take_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

void set_capturing(bool on)
{
    g_capturing = on;
    if (on) g_captured = 0;
}

void count_launch()
{
    if (g_capturing) ++g_captured;
    else g_launches.fetch_add(1, std::memory_order_relaxed);
}

uint64_t take_captured_launches()
{
    uint64_t c = g_captured;
    g_captured = 0;
    return c;
}

void prof_before(int kid, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on || g_capturing) return;
    g_pending_kid = kid;
    g_pending_a = take_event();
    cudaEventRecord(g_pending_a, s);
}

void prof_after(cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on || g_capturing || g_pending_kid < 0) return;
    cudaEvent_t b = take_event();
    cudaEventRecord(b, s);
    g_prof_recs.push_back({g_pending_kid, g_pending_a, b});
    g_pending_kid = -1;
    g_pending_a = nullptr;
}

const char* kernel_names[K_COUNT] = {
    "run_detect", "reverse", "tile_sort", "merge_partition", "merge_pass", "frog_plan", "frog_setup",
    "frog_partition", "frog_merge", "err_publish", "seg_plan", "seg_tile", "seg_merge", "learn_sample",
    "learn_fit", "learn_split", "learn_hist", "learn_scan", "learn_scatter", "learn_verify", "mlp_forward",
    "mlp_backward", "mlp_adam", "noalloc_sort", "learn_half_move"};

int num_sms()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 152;
    if (dev >= 0 && dev < 64) cached[dev] = v;
    return v;
}

namespace {
bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }
}  // namespace

int check_sort_args(const void* keys, const uint32_t* payload, int64_t n, int order, double bf)
{
    if (n < 0) return GNS_ERR_INVALID;
    if (order != GNS_ASCENDING && order != GNS_DESCENDING) return GNS_ERR_INVALID;
    if (isnan(bf) || bf < 0.0) return GNS_ERR_INVALID;
    if (n > 0 && keys == nullptr) return GNS_ERR_INVALID;
    if (keys && !aligned(keys, 8)) return GNS_ERR_INVALID;
    if (payload && !aligned(payload, 4)) return GNS_ERR_INVALID;
    if (n > 0 && payload) {
        const char* k0 = (const char*)keys;
        const char* k1 = k0 + (size_t)n * 8;
        const char* p0 = (const char*)payload;
        const char* p1 = p0 + (size_t)n * 4;
        if (p0 < k1 && k0 < p1) return GNS_ERR_INVALID;   // keys and payload overlap
    }
    if (bf < 1.0 / 64) return GNS_ERR_UNSUPPORTED;   // below Frogsort2's smallest inner fraction
    return GNS_OK;
}

}  // namespace gns

using namespace gns;

// ============================================================== C ABI
extern "C" {

static int mode_of(int key_type, int order)
{
    return (key_type == GNS_KEY_I64 ? MODE_I64 : 0) | (order == GNS_DESCENDING ? MODE_DESC : 0);
}

int gns_sort(double* keys, uint32_t* payload, int64_t n, int order, double buffer_fraction,
             gns_stream_t stream)
{
    int rc = check_sort_args(keys, payload, n, order, buffer_fraction);
    if (rc != GNS_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = sort_device((uint64_t*)keys, payload, n, mode_of(GNS_KEY_F64, order), buffer_fraction, s);
    return finish_call(rc, s);
}

int gns_sort_i64(int64_t* keys, uint32_t* payload, int64_t n, int order, double buffer_fraction,
                 gns_stream_t stream)
{
    int rc = check_sort_args(keys, payload, n, order, buffer_fraction);
    if (rc != GNS_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = sort_device((uint64_t*)keys, payload, n, mode_of(GNS_KEY_I64, order), buffer_fraction, s);
    return finish_call(rc, s);
}

int gns_sort_symmetric(void* keys, int key_type, uint32_t* payload, int64_t n, int order, double buffer_fraction,
                       int variant, gns_stream_t stream)
{
    if (key_type != GNS_KEY_F64 && key_type != GNS_KEY_I64) return GNS_ERR_INVALID;
    if (variant != GNS_FROGSORT1 && variant != GNS_GECKOSORT1 && variant != GNS_SQUIDSORT1) return GNS_ERR_INVALID;
    int rc = check_sort_args(keys, payload, n, order, buffer_fraction);   // NaN, negative, < 1/64
    if (rc != GNS_OK) return rc;
    if (buffer_fraction >= 1.0) return GNS_ERR_UNSUPPORTED;                 // no in-place layout at 100%
    cudaStream_t s = (cudaStream_t)stream;
    rc = sort_device_variant((uint64_t*)keys, payload, n, mode_of(key_type, order), buffer_fraction, variant, s);
    return finish_call(rc, s);
}

int gns_sort_host(void* keys_host, uint32_t* payload_host, int64_t n, int key_type, int order,
                  double buffer_fraction, gns_stream_t stream)
{
    if (key_type != GNS_KEY_F64 && key_type != GNS_KEY_I64) return GNS_ERR_INVALID;
    int rc = check_sort_args(keys_host, payload_host, n, order, buffer_fraction);
    if (rc != GNS_OK) return rc;
    if (n <= 1) return GNS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t kb = align256((size_t)n * 8), vb = payload_host ? align256((size_t)n * 4) : 0;
    char* d = (char*)ws_alloc(kb + vb, s);
    if (!d) return GNS_ERR_OOM;
    uint64_t* dk = (uint64_t*)d;
    uint32_t* dv = payload_host ? (uint32_t*)(d + kb) : nullptr;
    rc = GNS_ERR_CUDA;
    if (cudaMemcpyAsync(dk, keys_host, (size_t)n * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) goto out;
    if (dv && cudaMemcpyAsync(dv, payload_host, (size_t)n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        goto out;
    rc = sort_device(dk, dv, n, mode_of(key_type, order), buffer_fraction, s);
    if (rc != GNS_OK) goto out;
    rc = GNS_ERR_CUDA;
    if (cudaMemcpyAsync(keys_host, dk, (size_t)n * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) goto out;
    if (dv && cudaMemcpyAsync(payload_host, dv, (size_t)n * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        goto out;
    rc = GNS_OK;
out:
    ws_free(d, s);
    if (rc != GNS_OK) return rc;
    return gns_stream_status(stream);
}

size_t gns_workspace_bytes(int64_t n, double buffer_fraction, int kind)
{
    if (n < 0 || isnan(buffer_fraction)) return 0;
    if (kind == GNS_WS_SORT) return sort_workspace_bytes(n, buffer_fraction);
    if (kind == GNS_WS_LEARNED) return learned_workspace_bytes(n, buffer_fraction);
    return 0;
}

void gns_set_allocator(gns_alloc_fn alloc, gns_free_fn free_fn, void* ctx)
{
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = ctx;
}

int gns_stream_status(gns_stream_t stream)
{
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GNS_ERR_CUDA;
    int* p = status_word_ptr();
    if (!p) return GNS_ERR_CUDA;
    int v = 0, zero = 0;
    if (cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GNS_ERR_CUDA;
    if (v != 0 && cudaMemcpy(p, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return GNS_ERR_CUDA;
    return v;
}

const char* gns_strerror(int code)
{
    switch (code) {
        case GNS_OK: return "ok";
        case GNS_ERR_INVALID: return "invalid argument";
        case GNS_ERR_UNSUPPORTED: return "unsupported request";
        case GNS_ERR_OOM: return "workspace allocation failed";
        case GNS_ERR_CUDA: return "CUDA runtime error";
        case GNS_ERR_TIMEOUT: return "device-side wait timed out";
        case GNS_ERR_INTERNAL: return "device-side consistency check failed";
        default: return "unknown error";
    }
}

const char* gns_version(void) { return "gns 0.1.0 (sm_103a)"; }

uint64_t gns_launch_count(void) { return g_launches.load(); }

void gns_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
}

int gns_profile_read(int* kernel_ids, float* ms, int cap)
{
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        recs.swap(g_prof_recs);
    }
    int n = (int)recs.size();
    for (int i = 0; i < n; ++i) {
        cudaEventSynchronize(recs[i].b);
        float t = 0.f;
        cudaEventElapsedTime(&t, recs[i].a, recs[i].b);
        if (i < cap) {
            if (kernel_ids) kernel_ids[i] = recs[i].kid;
            if (ms) ms[i] = t;
        }
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : recs) {
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
    }
    return n;
}

const char* gns_kernel_name(int kernel_id)
{
    if (kernel_id < 0 || kernel_id >= K_COUNT) return "unknown";
    return kernel_names[kernel_id];
}

int gns_release_workspace_cache(void)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GNS_ERR_CUDA;
    cudaMemPool_t pool = workspace_pool(dev);
    if (!pool) return GNS_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return GNS_ERR_CUDA;
    return cudaMemPoolTrimTo(pool, 0) == cudaSuccess ? GNS_OK : GNS_ERR_CUDA;
}

void gns_set_wait_limit_ns(uint64_t ns) { g_wait_limit_ns.store(ns ? ns : 1); }

void gns_debug_skip_publish(int64_t ticket) { g_debug_skip.store(ticket); }
void gns_debug_jitter(uint32_t max_ns) { g_debug_jitter.store(max_ns > 50000u ? 50000u : max_ns); }

}  // extern "C"
