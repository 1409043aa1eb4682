// gns_noalloc.cu -- gns_sort_noalloc: the 100%-buffer stable sort for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they need a sort: real-time or signal-safe paths where an allocator call
// (which may lock, synchronise the device or map memory) is not allowed, hosts
// that reserve all device memory up front and hand a library only the buffers
// it works on, and code that runs under a fixed memory budget that leaves no
// room for the 12 bytes per element of scratch gns_sort takes.  This entry
// point sorts with no allocation at all: its scratch (the ping-pong buffer of
// the Nocopy merge levels, the merge-path splits and a few control words) is
// one file-scope device array of fixed size, GNS_NOALLOC_MAX_N elements' worth
// (about 12 MiB), which every GPU that loads this library holds until the
// process exits.  The passes are the ones gns_sort runs at the 100% tier
// (plain_sort_ext), so the two entry points cannot drift apart.
//
// The array's name is only a host-side stand-in for the device object: host
// code must never pass it to a kernel.  Its device address is fetched with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on that device, and cached.
#include <mutex>
#include <vector>

#include "gns_device.cuh"
#include "gns_internal.h"

namespace gns {

namespace {

constexpr int64_t kNoallocMaxN = GNS_NOALLOC_MAX_N;
constexpr size_t kCtlBytes = 256;
constexpr size_t kKeysBytes = (size_t)kNoallocMaxN * 8;
constexpr size_t kValsBytes = (size_t)kNoallocMaxN * 4;
// merge-path splits: one int64 per merge chunk; chunks hold at least 1024
// outputs, so this bounds plain_sort_splits(n) for every n <= the maximum
constexpr size_t kSplitBytes = ((size_t)(kNoallocMaxN / 1024) * 8 + 255) & ~(size_t)255;
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

}  // namespace

}  // namespace gns

using namespace gns;

extern "C" int gns_sort_noalloc(double* keys, uint32_t* payload, int64_t n, int order, gns_stream_t stream)
{
    int rc = check_sort_args(keys, payload, n, order, 1.0);   // includes the keys / payload overlap check
    if (rc != GNS_OK) return rc;
    if (n > kNoallocMaxN) return GNS_ERR_UNSUPPORTED;           // beyond the fixed scratch: use gns_sort
    if (n <= 1) return GNS_OK;
    if ((size_t)plain_sort_splits(n) * 8 > kSplitBytes) return GNS_ERR_INTERNAL;
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = scratch_ptr();
    if (!ws) return GNS_ERR_CUDA;
    const int mode = order == GNS_DESCENDING ? MODE_DESC : 0;
    // the array keeps the previous call's contents: plain_sort_ext resets the
    // control words; the buffer and the splits are written before they are read
    rc = plain_sort_ext((uint64_t*)keys, payload, n, mode, (uint64_t*)(ws + kCtlBytes),
                        payload ? (uint32_t*)(ws + kCtlBytes + kKeysBytes) : nullptr,
                        (int64_t*)(ws + kCtlBytes + kKeysBytes + kValsBytes), (int*)ws, nullptr, s);
    return finish_call(rc, s);
}
