// gns_internal.h -- host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "../../include/gns.h"

namespace gns {

// Kernel ids for instrumentation (gns_profile_read / gns_kernel_name).
enum KernelId {
    K_RUN_DETECT = 0,
    K_REVERSE,
    K_TILE_SORT,
    K_MERGE_PARTITION,
    K_MERGE_PASS,
    K_FROG_PLAN,
    K_FROG_SETUP,
    K_FROG_PARTITION,
    K_FROG_MERGE,
    K_ERR_PUBLISH,
    K_SEG_PLAN,
    K_SEG_TILE,
    K_SEG_MERGE,
    K_LEARN_SAMPLE,
    K_LEARN_FIT,
    K_LEARN_SPLIT,
    K_LEARN_HIST,
    K_LEARN_SCAN,
    K_LEARN_SCATTER,
    K_LEARN_VERIFY,
    K_MLP_FWD,
    K_MLP_BWD,
    K_MLP_ADAM,
    K_NOALLOC_SORT,
    K_LEARN_HALF,
    K_COUNT
};

// Launch bookkeeping: count every launch; when profiling is on, bracket it by
// events on its stream.
void prof_before(int kid, cudaStream_t s);
void prof_after(cudaStream_t s);
extern std::atomic<uint64_t> g_launches;
// While a graph is being captured on this thread, launches are counted into the
// graph (and added to g_launches each time the graph is launched) and not
// bracketed by profiling events.
void set_capturing(bool on);
void count_launch();
uint64_t take_captured_launches();

template <typename Kernel, typename... Args>
inline cudaError_t launch(int kid, Kernel kernel, dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s, Args... args)
{
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
    prof_before(kid, s);
    kernel<<<grid, block, smem, s>>>(args...);
    cudaError_t e = cudaGetLastError();
    prof_after(s);
    count_launch();
    return e;
}

// Device address of the per-device status word (resolved once per device).
int* status_word_ptr();

// Scratch allocation through the allocator hook.
void* ws_alloc(size_t bytes, cudaStream_t s);
void ws_free(void* p, cudaStream_t s);

// Spin limit of bounded device waits, and the debug fault switch.
uint64_t wait_limit_ns();
int64_t take_debug_skip_publish();   // returns the ticket (or -1) and clears it
uint32_t debug_jitter_ns();           // test hook: bounded random delay before in-place loads (0 = off)

// Folds a call's error word into the per-device status word (one tiny kernel).
cudaError_t publish_call_error(const int* call_err, cudaStream_t s);

// GNS_SYNC_STATUS=1: synchronise and return the status word after each call.
int finish_call(int rc, cudaStream_t s);

// Rounds a byte count up to 256 (every workspace sub-buffer starts aligned).
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Runs f() once for each device ordinal it is called on (with that device
// current): function attributes such as the dynamic shared-memory limit belong
// to the context of the device that was current when they were set.
struct PerDeviceOnce {
    std::mutex mu;
    bool done[64] = {};
    template <typename F>
    void run(F f)
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && done[dev]) return;
        f();
        if (dev >= 0 && dev < 64) done[dev] = true;
    }
};

// Host-side argument checks shared by the sorting entry points: n >= 0, a
// known order, a non-negative buffer fraction, non-NULL aligned keys when
// n > 0, an aligned payload that does not overlap the keys.
int check_sort_args(const void* keys, const uint32_t* payload, int64_t n, int order, double bf);

// Number of SMs of the current device (cached per device).
int num_sms();

// gns_sort core: keys are raw 64-bit patterns, mode = key type | order bits.
int sort_device(uint64_t* keys, uint32_t* payload, int64_t n, int mode,
                double buffer_fraction, cudaStream_t s);
// sort_device with a symmetric variant of the in-place tiers (bf < 1): 0 =
// Frogsort, 1 = Geckosort, 2 = Squidsort (gns_sort_symmetric).
int sort_device_variant(uint64_t* keys, uint32_t* payload, int64_t n, int mode, double buffer_fraction,
                        int variant, cudaStream_t s);

// The 100% tier (tile sort, then Nocopy merge levels) on scratch the caller
// provides: bufk / bufv hold n keys / n payloads (bufv unused without a
// payload), splits holds plain_sort_splits(n) int64 words, ctl 256 bytes of
// control words (reset by the call).  gate == nullptr: a run-detection pass
// comes first (presorted input costs one read, strictly descending input one
// reversal).  gate != nullptr: a device int read when the sort starts; every
// kernel of the sort returns at once unless it is non-zero, so that whether the
// sort runs is decided on the device.  Returns GNS_OK or GNS_ERR_CUDA.
int plain_sort_ext(uint64_t* keys, uint32_t* vals, int64_t n, int mode, uint64_t* bufk, uint32_t* bufv,
                   int64_t* splits, int* ctl, const int* gate, cudaStream_t s);
int64_t plain_sort_splits(int64_t n);
size_t sort_workspace_bytes(int64_t n, double buffer_fraction);

// Segmented sort core and helpers (gns_segmented.cu).
int segmented_sort_device(uint64_t* keys, uint32_t* vals, const int64_t* off, int64_t nseg, int64_t n, int mode,
                          cudaStream_t s);
size_t segmented_workspace_bytes(int64_t n, int64_t nseg, bool ext_buf = false);
int ordered_sort_direct(uint64_t* keys, uint32_t* vals, const int64_t* off, int64_t nseg, int64_t n, int mode,
                        const uint8_t* skip, cudaStream_t s, uint64_t* xbufk = nullptr, uint32_t* xbufv = nullptr);
size_t learned_workspace_bytes(int64_t n, double buffer_fraction);

}  // namespace gns
