// gns_noalloc.cu -- gns_sort_noalloc: the 100%-buffer stable sort for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they need a sort: code running while a CUDA graph is being captured by
// someone else, real-time or signal-safe paths that forbid allocation, or
// embedding environments that own all device memory and give a library only
// the buffers it is handed.  This entry point sorts with no allocation at all:
// its scratch (the ping-pong buffer of the Nocopy merge levels, the merge-path
// splits and a few control words) is one file-scope device array of fixed
// size, GNS_NOALLOC_MAX_N elements' worth (about 12 MiB), which every GPU that
// loads this library holds until the process exits.
//
// The array's name is only a host-side stand-in for the device object: host
// code must never pass it to a kernel.  Its device address is fetched with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on that device, and cached.
#include <mutex>
#include <vector>

#include "gns_internal.h"
#include "gns_kernels.cuh"
#include "gns_merge_tma.cuh"
#include "gns_merge_ws.cuh"

namespace gns {

namespace {

constexpr int64_t kNoallocMaxN = GNS_NOALLOC_MAX_N;
constexpr size_t kCtlBytes = 256;
constexpr size_t kKeysBytes = (size_t)kNoallocMaxN * 8;
constexpr size_t kValsBytes = (size_t)kNoallocMaxN * 4;
constexpr size_t kSplitBytes = ((size_t)(kNoallocMaxN / CHUNK) * 8 + 255) & ~(size_t)255;
constexpr size_t kScratchBytes = kCtlBytes + kKeysBytes + kValsBytes + kSplitBytes;

// Shared by every call on a device: calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_scratch_mu;
std::vector<char*> g_scratch_ptrs;   // device address per device ordinal

// Device address of the scratch array on the current device (nullptr on error).
char* scratch_ptr()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if ((int)g_scratch_ptrs.size() <= dev) g_scratch_ptrs.resize(dev + 1, nullptr);
    if (!g_scratch_ptrs[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_ptrs[dev] = (char*)p;
    }
    return g_scratch_ptrs[dev];
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

std::once_flag g_attr_once;
void init_attributes()
{
    std::call_once(g_attr_once, [] {
        cudaFuncSetAttribute(tile_sort_kernel<SORT_THREADS, SORT_ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SmemKV<TILE>));
        cudaFuncSetAttribute(merge_pass_ws_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(WsSmemOut<WS_CHUNK, 2>));
    });
}

int sms()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 152;
}

}  // namespace

}  // namespace gns

using namespace gns;

extern "C" int gns_sort_noalloc(double* keys, uint32_t* payload, int64_t n, int order, gns_stream_t stream)
{
    if (n < 0 || (order != GNS_ASCENDING && order != GNS_DESCENDING)) return GNS_ERR_INVALID;
    if (n > 0 && keys == nullptr) return GNS_ERR_INVALID;
    if (((uintptr_t)keys & 7) || ((uintptr_t)payload & 3)) return GNS_ERR_INVALID;
    if (n > kNoallocMaxN) return GNS_ERR_UNSUPPORTED;           // beyond the fixed scratch
    if (n <= 1) return GNS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = scratch_ptr();
    if (!ws) return GNS_ERR_CUDA;
    init_attributes();
    const int mode = order == GNS_DESCENDING ? MODE_DESC : 0;
    uint64_t* k = (uint64_t*)keys;
    uint32_t* v = payload;
    int* ctl = (int*)ws;
    int* presorted = ctl;
    int* call_err = ctl + 2;
    uint64_t* bufk = (uint64_t*)(ws + kCtlBytes);
    uint32_t* bufv = v ? (uint32_t*)(ws + kCtlBytes + kKeysBytes) : nullptr;
    int64_t* splits = (int64_t*)(ws + kCtlBytes + kKeysBytes + kValsBytes);
    int* status = status_word_ptr();
    if (!status) return GNS_ERR_CUDA;

    // the array keeps the previous call's contents: reset the control words
    if (cudaMemsetAsync(ctl, 0, kCtlBytes, s) != cudaSuccess) return GNS_ERR_CUDA;
    if (cudaMemsetAsync(presorted, 1, 2 * sizeof(int), s) != cudaSuccess) return GNS_ERR_CUDA;
    cudaError_t e = launch(K_NOALLOC_SORT, run_detect_kernel, dim3((unsigned)ceil_div(n, DETECT_TILE)), dim3(256), 0,
                           s, (const uint64_t*)k, n, mode, presorted);
    if (e == cudaSuccess)
        e = launch(K_NOALLOC_SORT, reverse_kernel, dim3(152 * 8), dim3(256), 0, s, k, v, n, (const int*)presorted);
    int levels = 0;
    while ((1ll << levels) < ceil_div(n, TILE)) ++levels;
    uint64_t* cur_k = (levels & 1) ? bufk : k;
    uint32_t* cur_v = (levels & 1) ? bufv : v;
    uint64_t* oth_k = (levels & 1) ? k : bufk;
    uint32_t* oth_v = (levels & 1) ? v : bufv;
    if (e == cudaSuccess)
        e = launch(K_NOALLOC_SORT, tile_sort_kernel<SORT_THREADS, SORT_ITEMS>, dim3((unsigned)ceil_div(n, TILE)),
                   dim3(SORT_THREADS), sizeof(SmemKV<TILE>), s, (const uint64_t*)k, (const uint32_t*)v, cur_k, cur_v,
                   n, mode, (int)(levels == 0), (const int*)presorted);
    const int64_t nblocks = ceil_div(n, CHUNK);
    for (int lvl = 0; lvl < levels && e == cudaSuccess; ++lvl) {
        const int64_t w = (int64_t)TILE << lvl;
        e = launch(K_NOALLOC_SORT, merge_partition_kernel, dim3((unsigned)ceil_div(nblocks, 256)), dim3(256), 0, s,
                   (const uint64_t*)cur_k, n, w, nblocks, splits, (const int*)presorted);
        if (e != cudaSuccess) break;
        const int64_t cap = (int64_t)sms() * ws_ctas_per_sm<2>();
        const int64_t grid = nblocks < cap ? nblocks : cap;
        e = launch(K_NOALLOC_SORT, merge_pass_ws_kernel<2>, dim3((unsigned)grid), dim3(WS_CONSUMERS + 32),
                   sizeof(WsSmemOut<WS_CHUNK, 2>), s, (const uint64_t*)cur_k, (const uint32_t*)cur_v, oth_k, oth_v, n,
                   w, nblocks, (const int64_t*)splits, mode, (int)(lvl == levels - 1), call_err, wait_limit_ns(),
                   (const int*)presorted);
        uint64_t* tk = cur_k; cur_k = oth_k; oth_k = tk;
        uint32_t* tv = cur_v; cur_v = oth_v; oth_v = tv;
    }
    if (e == cudaSuccess)
        e = launch(K_NOALLOC_SORT, publish_err_kernel, dim3(1), dim3(1), 0, s, (const int*)call_err, status);
    return finish_call(e == cudaSuccess ? GNS_OK : GNS_ERR_CUDA, s);
}
