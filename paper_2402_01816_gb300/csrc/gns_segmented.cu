// gns_segmented.cu -- batched segmented stable sort (no counterpart in the paper:
// a batching form of the same mergesort).
//
// Every segment [offsets[s], offsets[s+1]) is sorted independently, all of them
// in one CUDA-graph launch:
//   plan      per segment: tiles, merge levels k_s = ceil(log2(#tiles)), and the
//             number of merge chunks it contributes to each level; one exclusive
//             scan per row gives every kernel its work list on the device.
//   tiles     size classes: segments up to the small-class bound are sorted by a
//             smaller CTA shape (one tile each); all other segments are cut into
//             4096-element tiles.  A segment with an odd number of levels writes
//             its tiles to the buffer, so that its last level lands in `keys`
//             (the merge decides where the data lies, as Omitsort does in the
//             "Full adaptivity" section); a one-tile segment is done here.
//   levels    level p merges the segments with k_s > p only: a partition kernel
//             writes each 1024-output chunk's slices, the TMA merge pipeline of
//             the plain sort consumes the list.
// The whole sequence is captured once per (pointers, sizes, order, stream's
// device, tuned schedule) and replayed; the tuned schedule (small-class bound
// and its CTA shape) is picked by timing the candidates on a scratch copy the
// first time a shape is seen.
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "gns_internal.h"
#include "gns_kernels.cuh"
#include "gns_merge_tma.cuh"
#include "gns_merge_ws.cuh"

namespace gns {

namespace {

constexpr int SEG_T_MIN = 4096;    // smallest big-class tile (seg_tile_kernel<256, 16>); 8192 with <512, 16>

struct SegChunk {
    int64_t out0, a_src, b_src;    // absolute positions
    int32_t na, nb;
    int32_t flags;                 // bit 0: read the buffer (else keys); bit 1: last level (decode)
    int32_t pad;
};

// ---------------------------------------------------------------- plan
// rows (each nseg + 1 long): row 0 = small-class tiles, row 1 = big-class tiles,
// row 2 + p = merge chunks of level p.
__global__ void seg_count_kernel(const int64_t* __restrict__ off, int64_t nseg, int L, int64_t small_max,
                                 int64_t big_t, int64_t* rows, uint8_t* levels, const int* ctl)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg || skip_all(ctl)) return;
    const int64_t stride = nseg + 1;
    const int64_t len = off[s + 1] - off[s];
    const int64_t tiles = (len + big_t - 1) / big_t;
    int k = 0;
    while ((1ll << k) < tiles) ++k;
    levels[s] = (uint8_t)k;
    const bool small = len > 0 && len <= small_max;
    rows[s] = small ? 1 : 0;
    rows[stride + s] = small ? 0 : tiles;
    const int64_t chunks = (len + CHUNK - 1) / CHUNK;
    for (int p = 0; p < L; ++p) rows[(2 + p) * stride + s] = k > p ? chunks : 0;
}

// Exclusive scan of row blockIdx.x in place; the total goes to entry nseg.
__global__ void __launch_bounds__(1024) seg_scan_kernel(int64_t* rows, int64_t nseg, const int* ctl)
{
    if (skip_all(ctl)) return;
    __shared__ int64_t warp_sum[32];
    __shared__ int64_t s_carry;
    int64_t* row = rows + (int64_t)blockIdx.x * (nseg + 1);
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nseg; base += 1024) {
        const int64_t i = base + t;
        const int64_t v = i < nseg ? row[i] : 0;
        int64_t x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) warp_sum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int64_t w = warp_sum[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += y;
            }
            warp_sum[lane] = w;                 // inclusive over warps
        }
        __syncthreads();
        const int64_t incl = x + (wid > 0 ? warp_sum[wid - 1] : 0);
        const int64_t carry = s_carry;
        if (i < nseg) row[i] = carry + incl - v;
        __syncthreads();
        if (t == 1023) s_carry = carry + incl;
        __syncthreads();
    }
    if (t == 0) row[nseg] = s_carry;
}

// Largest s in [0, nseg) with prefix[s] <= i (prefix non-decreasing, i < prefix[nseg]).
__device__ __forceinline__ int64_t seg_of(const int64_t* prefix, int64_t nseg, int64_t i)
{
    int64_t lo = 0, hi = nseg - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- tiles
// Persistent: work item i of the row = tile (i - prefix[s]) of segment s.
// big == 0: the row counts one tile per small segment (sorted whole).
template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)   // <= 64 registers: 1024 threads per SM
    seg_tile_kernel(uint64_t* keys, uint32_t* vals, uint64_t* bufk, uint32_t* bufv, const int64_t* __restrict__ off,
                    int64_t nseg, const int64_t* __restrict__ prefix, const uint8_t* __restrict__ levels, int mode,
                    const int* ctl)
{
    constexpr int T = THREADS * ITEMS;
    if (skip_all(ctl)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemKV<T>& sm = *reinterpret_cast<SmemKV<T>*>(smem_raw);
    __shared__ int64_t s_base, s_seg_end;
    __shared__ int s_k;
    const int t = threadIdx.x;
    const int64_t total = prefix[nseg];
    for (int64_t i = blockIdx.x; i < total; i += gridDim.x) {
        if (t == 0) {
            const int64_t s = seg_of(prefix, nseg, i);
            s_base = off[s] + (i - prefix[s]) * T;
            s_seg_end = off[s + 1];
            s_k = levels[s];
        }
        __syncthreads();
        const int64_t base = s_base;
        const int nv = (int)imin64(T, s_seg_end - base);
        const int k = s_k;
#pragma unroll 4
        for (int j = 0; j < ITEMS; ++j) {
            int e = t + j * THREADS;
            bool ok = e < nv;
            sm.k[pidx(e)] = ok ? encode_key(keys[base + e], mode) : ~0ull;
            sm.v[pidx(e)] = (ok && vals) ? vals[base + e] : 0u;
        }
        block_sort_smem<THREADS, ITEMS>(sm, nv);
        uint64_t* dk = (k & 1) ? bufk : keys;
        uint32_t* dv = (k & 1) ? bufv : vals;
#pragma unroll 4
        for (int j = 0; j < ITEMS; ++j) {
            int e = t + j * THREADS;
            if (e < nv) {
                uint64_t key = sm.k[pidx(e)];
                dk[base + e] = k == 0 ? decode_key(key, mode) : key;
                if (dv) dv[base + e] = sm.v[pidx(e)];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- levels
// One thread per work item of level p: its segment, its chunk and both
// merge-path splits, written to list[i].
__global__ void seg_partition_kernel(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ bufk,
                                     const int64_t* __restrict__ off, int64_t nseg, const int64_t* __restrict__ prefix,
                                     const uint8_t* __restrict__ levels, int p, int64_t big_t, SegChunk* list,
                                     const int* ctl)
{
    if (skip_all(ctl)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= prefix[nseg]) return;
    const int64_t s = seg_of(prefix, nseg, i);
    const int64_t c = i - prefix[s];
    const int64_t seg0 = off[s], len = off[s + 1] - seg0;
    const int k = levels[s];
    const int from_buf = (k - p) & 1;
    const uint64_t* src = (from_buf ? bufk : keys) + seg0;
    const int64_t w = big_t << p;
    const int64_t o = c * CHUNK;
    const int64_t ps = (o / (2 * w)) * (2 * w);
    const int64_t lenA = imin64(w, len - ps), lenB = imax64(0, imin64(w, len - ps - w));
    const int64_t d0 = o - ps, d1 = imin64(d0 + CHUNK, lenA + lenB);
    const uint64_t* A = src + ps;
    const uint64_t* B = A + lenA;
    auto ga = [&](int64_t x) { return A[x]; };
    auto gb = [&](int64_t x) { return B[x]; };
    const int64_t a0 = merge_path(d0, lenA, lenB, ga, gb);
    const int64_t a1 = merge_path(d1, lenA, lenB, ga, gb);
    SegChunk r;
    r.out0 = seg0 + o;
    r.a_src = seg0 + ps + a0;
    r.b_src = seg0 + ps + lenA + (d0 - a0);
    r.na = (int32_t)(a1 - a0);
    r.nb = (int32_t)((d1 - a1) - (d0 - a0));
    r.flags = from_buf | ((p == k - 1) ? 2 : 0);
    r.pad = 0;
    list[i] = r;
}

// One merge level of the segmented sort, chunk list from seg_partition_kernel,
// through the warp-specialised pipeline of the plain levels: item i of the
// list goes to CTA i mod gridDim.x.
struct SegLevelSrc {
    uint64_t* keys; uint32_t* vals; uint64_t* bufk; uint32_t* bufv;
    int64_t n;
    const SegChunk* list;
    int64_t count, i;
    __device__ __forceinline__ bool next(WsLoad& L)
    {
        if (i >= count) return false;
        const SegChunk r = list[i];
        i += gridDim.x;
        const bool fb = r.flags & 1;
        const uint64_t* sk = fb ? bufk : keys;
        const uint32_t* sv = fb ? bufv : vals;
        uint64_t* dk = fb ? keys : bufk;
        uint32_t* dv = fb ? vals : bufv;
        L.ak = sk + r.a_src; L.av = sv ? sv + r.a_src : nullptr; L.na = r.na;
        L.bk = sk + r.b_src; L.bv = sv ? sv + r.b_src : nullptr; L.nb = r.nb;
        L.ak_end = L.bk_end = sk + n;
        L.av_end = L.bv_end = sv ? sv + n : nullptr;
        L.plain_a = L.plain_b = false;
        L.slot_a = L.slot_b = 0;
        L.dk = dk + r.out0; L.dv = dv ? dv + r.out0 : nullptr;
        L.oslot = 0;
        L.decode = (r.flags >> 1) & 1;
        L.tk = 0;
        L.dep_lo = 0;
        L.dep_hi = -1;
        return true;
    }
};

constexpr int SEG_WS_STAGES = 2;

__global__ void __launch_bounds__(WS_CONSUMERS + 32, ws_ctas_per_sm<SEG_WS_STAGES>())
    seg_merge_ws_kernel(uint64_t* keys, uint32_t* vals, uint64_t* bufk, uint32_t* bufv, int64_t n,
                        const SegChunk* __restrict__ list, const int64_t* __restrict__ count, int mode, int* call_err,
                        uint64_t limit_ns, const int* ctl)
{
    if (skip_all(ctl)) return;
    const int64_t cnt = *count;
    if ((int64_t)blockIdx.x >= cnt) return;
    SegLevelSrc src{keys, vals, bufk, bufv, n, list, cnt, (int64_t)blockIdx.x};
    ws_merge_out<WS_CONSUMERS, WS_ITEMS, SEG_WS_STAGES>(src, vals != nullptr, mode, call_err, limit_ns);
}

// ---------------------------------------------------------------- ordered segments
// Segments whose key ranges are ordered (every key of segment s lies at or
// below every key of segment s + 1, and equal keys share a segment: the
// learned sort's buckets).  Sorting any range that holds whole parts of
// several such segments keeps each part in its own positions, so the array is
// tile-sorted at the global ORD_T-key tiles, each tile sorted whole whatever
// segment ends it holds, and each segment is finished by merge levels over its
// own runs.  With a = floor(s0 / ORD_T) * ORD_T for a segment starting at s0,
// run j covers [a + j ORD_T, a + (j + 1) ORD_T) clipped to the segment (run 0
// its head inside the first tile, the last its tail); level p merges runs in
// pairs of 2^p, aligned to a, so the segment needs ceil(log2(tiles it
// touches)) levels, and chunks of CHUNK outputs aligned to a never straddle
// a pair.  The data lands in `keys` after a segment's last level (its tiles go
// to the buffer when its level count is odd).
constexpr int64_t ORD_T = 8192;

// Largest s in [lo, hi] with off[s] <= pos (off non-decreasing; off[lo] <= pos).
__device__ __forceinline__ int64_t seg_at(const int64_t* __restrict__ off, int64_t lo, int64_t hi, int64_t pos)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(&off[mid]) <= pos) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Per segment: its level count and, for every level p < L, the chunks it
// contributes (rows[p * (nseg + 1) + s]).  A segment flagged in skip (all
// keys equal) or empty gets no level.
__global__ void ord_count_kernel(const int64_t* __restrict__ off, int64_t nseg, int L, int64_t* rows,
                                 uint8_t* levels, const uint8_t* __restrict__ skip, const int* ctl)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg || skip_all(ctl)) return;
    const int64_t stride = nseg + 1;
    const int64_t s0 = off[s], s1 = off[s + 1];
    int k = 0;
    int64_t chunks = 0;
    if (s1 > s0 && !(skip && skip[s])) {
        const int64_t a = s0 / ORD_T * ORD_T;
        const int64_t tiles = (s1 - 1 - a) / ORD_T + 1;
        while ((1ll << k) < tiles) ++k;
        chunks = (s1 - 1 - a) / CHUNK - (s0 - a) / CHUNK + 1;
    }
    levels[s] = (uint8_t)k;
    for (int p = 0; p < L; ++p) rows[p * stride + s] = k > p ? chunks : 0;
}

// One CTA per global tile: the tile is sorted whole, and every output goes to
// the buffer or to `keys` by its segment's level count (odd: buffer), decoded
// when the segment has no level.  A tile inside one skipped segment is left
// as it is.
template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)   // <= 64 registers: 1024 threads per SM
    ord_tile_kernel(uint64_t* keys, uint32_t* vals, uint64_t* bufk, uint32_t* bufv, int64_t n,
                    const int64_t* __restrict__ off, int64_t nseg, const uint8_t* __restrict__ levels,
                    const uint8_t* __restrict__ skip, int mode, const int* ctl)
{
    constexpr int T = THREADS * ITEMS;
    static_assert(T == ORD_T, "tile");
    if (skip_all(ctl)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemKV<T>& sm = *reinterpret_cast<SmemKV<T>*>(smem_raw);
    __shared__ int64_t s_first, s_last;
    const int t = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * T;
    const int nv = (int)imin64(T, n - base);
    if (t == 0) {
        s_first = seg_at(off, 0, nseg - 1, base);
        s_last = seg_at(off, s_first, nseg - 1, base + nv - 1);
    }
    __syncthreads();
    const int64_t sf = s_first, sl = s_last;
    if (sf == sl && skip && skip[sf]) return;
#pragma unroll 4
    for (int j = 0; j < ITEMS; ++j) {
        const int e = t + j * THREADS;
        const bool ok = e < nv;
        sm.k[pidx(e)] = ok ? encode_key(keys[base + e], mode) : ~0ull;
        sm.v[pidx(e)] = (ok && vals) ? vals[base + e] : 0u;
    }
    block_sort_smem<THREADS, ITEMS>(sm, nv);
    const int k_one = levels[sf];
#pragma unroll 4
    for (int j = 0; j < ITEMS; ++j) {
        const int e = t + j * THREADS;
        if (e < nv) {
            const int k = sf == sl ? k_one : (int)__ldg(&levels[seg_at(off, sf, sl, base + e)]);
            const uint64_t key = sm.k[pidx(e)];
            ((k & 1) ? bufk : keys)[base + e] = k == 0 ? decode_key(key, mode) : key;
            if (vals) ((k & 1) ? bufv : vals)[base + e] = sm.v[pidx(e)];
        }
    }
}

// One thread per work item of level p: its segment, its chunk and both
// merge-path splits, as absolute positions, written to list[i].
__global__ void ord_partition_kernel(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ bufk,
                                     const int64_t* __restrict__ off, int64_t nseg, const int64_t* __restrict__ prefix,
                                     const uint8_t* __restrict__ levels, int p, SegChunk* list, const int* ctl)
{
    if (skip_all(ctl)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= prefix[nseg]) return;
    const int64_t s = seg_of(prefix, nseg, i);
    const int64_t s0 = off[s], s1 = off[s + 1];
    const int64_t a = s0 / ORD_T * ORD_T;
    const int k = levels[s];
    const int from_buf = (k - p) & 1;
    const uint64_t* src = from_buf ? bufk : keys;
    const int64_t w = ORD_T << p;
    const int64_t c = (s0 - a) / CHUNK + (i - prefix[s]);      // chunk index counted from a
    const int64_t o0 = imax64(s0, a + c * CHUNK), o1 = imin64(s1, a + (c + 1) * CHUNK);
    const int64_t pair_lo = a + (c * CHUNK) / (2 * w) * (2 * w), pair_mid = pair_lo + w, pair_hi = pair_mid + w;
    const int64_t pa0 = imax64(s0, pair_lo), pa1 = imin64(s1, pair_mid);
    const int64_t pb0 = imin64(imax64(s0, pair_mid), s1), pb1 = imin64(s1, pair_hi);   // empty B: at s1
    const int64_t lenA = imax64(0, pa1 - pa0), lenB = imax64(0, pb1 - pb0);
    const int64_t d0 = o0 - pa0, d1 = o1 - pa0;                 // the pair's outputs start at pa0
    const uint64_t* A = src + pa0;
    const uint64_t* B = src + pb0;
    auto ga = [&](int64_t x) { return A[x]; };
    auto gb = [&](int64_t x) { return B[x]; };
    const int64_t a0 = merge_path(d0, lenA, lenB, ga, gb);
    const int64_t a1 = merge_path(d1, lenA, lenB, ga, gb);
    SegChunk r;
    r.out0 = o0;
    r.a_src = pa0 + a0;
    r.b_src = pb0 + (d0 - a0);
    r.na = (int32_t)(a1 - a0);
    r.nb = (int32_t)((d1 - a1) - (d0 - a0));
    r.flags = from_buf | ((p == k - 1) ? 2 : 0);
    r.pad = 0;
    list[i] = r;
}

// ---------------------------------------------------------------- host side
int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int num_sms_dev()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 152;
}

// Schedules the autotuner chooses from: small-class bound and its CTA shape,
// and the big class's tile (4096 keys by 256 threads or 8192 by 512).
struct SegSchedule {
    int64_t small_max;   // 0: no small class
    int small_threads;   // 64 (x16 = 1024 keys) or 128 (x16 = 2048 keys)
    int big_t;           // 4096 or 8192
};
const SegSchedule kCandidates[] = {{0, 0, 4096}, {1024, 64, 4096}, {2048, 128, 4096}, {0, 0, 8192},
                                   {2048, 128, 8192}};

int max_levels(int64_t n)
{
    int64_t tiles = ceil_div(n, SEG_T_MIN);
    int L = 0;
    while ((1ll << L) < tiles) ++L;
    return L;
}

struct SegLayout {
    size_t ctl, bufk, bufv, rows, levels, list, total;
    int L;
    int64_t max_items;
};

// ext_buf: the caller provides the n-element ping-pong buffer, which is then
// not part of the workspace.
SegLayout seg_layout(int64_t n, int64_t nseg, bool with_vals, bool ext_buf = false)
{
    SegLayout o{};
    size_t off = 0;
    o.L = max_levels(n);
    o.max_items = ceil_div(n, CHUNK) + nseg;
    o.ctl = off; off += 256;
    o.bufk = off; off += ext_buf ? 0 : align256((size_t)n * 8);
    o.bufv = off; off += (with_vals && !ext_buf) ? align256((size_t)n * 4) : 0;
    o.rows = off; off += align256((size_t)(2 + o.L) * (size_t)(nseg + 1) * 8);
    o.levels = off; off += align256((size_t)nseg);
    o.list = off; off += align256((size_t)o.max_items * sizeof(SegChunk));
    o.total = off;
    return o;
}

PerDeviceOnce g_seg_attr_once;
void seg_init_attributes()
{
    g_seg_attr_once.run([] {
        cudaFuncSetAttribute(seg_tile_kernel<256, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SmemKV<4096>));
        cudaFuncSetAttribute(seg_tile_kernel<512, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SmemKV<8192>));
        cudaFuncSetAttribute(seg_tile_kernel<128, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SmemKV<2048>));
        cudaFuncSetAttribute(seg_tile_kernel<64, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SmemKV<1024>));
        cudaFuncSetAttribute(seg_merge_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(WsSmemOut<WS_CHUNK, SEG_WS_STAGES>));
        cudaFuncSetAttribute(ord_tile_kernel<512, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SmemKV<8192>));
    });
}

// Enqueues the whole segmented sort on s (keys/vals in place, ws laid out by lay).
cudaError_t seg_enqueue(uint64_t* keys, uint32_t* vals, const int64_t* off, int64_t nseg, int64_t n, int mode,
                        const SegSchedule& sch, char* ws, const SegLayout& lay, cudaStream_t s)
{
    int* ctl = (int*)(ws + lay.ctl);
    int* call_err = ctl + 2;
    uint64_t* bufk = (uint64_t*)(ws + lay.bufk);
    uint32_t* bufv = vals ? (uint32_t*)(ws + lay.bufv) : nullptr;
    int64_t* rows = (int64_t*)(ws + lay.rows);
    uint8_t* levels = (uint8_t*)(ws + lay.levels);
    SegChunk* list = (SegChunk*)(ws + lay.list);
    const int64_t stride = nseg + 1;
    const int sms = num_sms_dev();
    cudaError_t e = cudaMemsetAsync(ctl, 0, 256, s);
    if (e != cudaSuccess) return e;
    e = launch(K_SEG_PLAN, seg_count_kernel, dim3((unsigned)ceil_div(nseg, 256)), dim3(256), 0, s, off, nseg, lay.L,
               sch.small_max, (int64_t)sch.big_t, rows, levels, (const int*)ctl);
    if (e != cudaSuccess) return e;
    e = launch(K_SEG_PLAN, seg_scan_kernel, dim3((unsigned)(2 + lay.L)), dim3(1024), 0, s, rows, nseg,
               (const int*)ctl);
    if (e != cudaSuccess) return e;
    if (sch.small_max > 0) {
        if (sch.small_threads == 64)
            e = launch(K_SEG_TILE, seg_tile_kernel<64, 16>, dim3((unsigned)(sms * 8)), dim3(64), sizeof(SmemKV<1024>),
                       s, keys, vals, bufk, bufv, off, nseg, (const int64_t*)rows, (const uint8_t*)levels, mode,
                       (const int*)ctl);
        else
            e = launch(K_SEG_TILE, seg_tile_kernel<128, 16>, dim3((unsigned)(sms * 8)), dim3(128),
                       sizeof(SmemKV<2048>), s, keys, vals, bufk, bufv, off, nseg, (const int64_t*)rows,
                       (const uint8_t*)levels, mode, (const int*)ctl);
        if (e != cudaSuccess) return e;
    }
    if (sch.big_t == 8192)
        e = launch(K_SEG_TILE, seg_tile_kernel<512, 16>, dim3((unsigned)(sms * 2)), dim3(512), sizeof(SmemKV<8192>),
                   s, keys, vals, bufk, bufv, off, nseg, (const int64_t*)(rows + stride), (const uint8_t*)levels, mode,
                   (const int*)ctl);
    else
        e = launch(K_SEG_TILE, seg_tile_kernel<256, 16>, dim3((unsigned)(sms * 4)), dim3(256), sizeof(SmemKV<4096>),
                   s, keys, vals, bufk, bufv, off, nseg, (const int64_t*)(rows + stride), (const uint8_t*)levels, mode,
                   (const int*)ctl);
    if (e != cudaSuccess) return e;
    for (int p = 0; p < lay.L; ++p) {
        const int64_t* prefix = rows + (2 + p) * stride;
        e = launch(K_SEG_MERGE, seg_partition_kernel, dim3((unsigned)ceil_div(lay.max_items, 256)), dim3(256), 0, s,
                   (const uint64_t*)keys, (const uint64_t*)bufk, off, nseg, prefix, (const uint8_t*)levels, p,
                   (int64_t)sch.big_t, list, (const int*)ctl);
        if (e != cudaSuccess) return e;
        const int64_t cap = (int64_t)sms * ws_ctas_per_sm<SEG_WS_STAGES>();
        const int64_t grid = lay.max_items < cap ? lay.max_items : cap;
        e = launch(K_SEG_MERGE, seg_merge_ws_kernel, dim3((unsigned)grid), dim3(WS_CONSUMERS + 32),
                   sizeof(WsSmemOut<WS_CHUNK, SEG_WS_STAGES>), s, keys, vals, bufk, bufv, n, (const SegChunk*)list,
                   (const int64_t*)(prefix + nseg), mode, call_err, wait_limit_ns(), (const int*)ctl);
        if (e != cudaSuccess) return e;
    }
    return publish_call_error(call_err, s);
}

// Enqueues the sort of ordered segments on s (keys/vals in place, ws laid out
// by seg_layout; rows 0 .. L-1 of it hold the level rows).
cudaError_t ord_enqueue(uint64_t* keys, uint32_t* vals, const int64_t* off, int64_t nseg, int64_t n, int mode,
                        char* ws, const SegLayout& lay, cudaStream_t s, const uint8_t* skip, uint64_t* xbufk,
                        uint32_t* xbufv)
{
    int* ctl = (int*)(ws + lay.ctl);
    int* call_err = ctl + 2;
    uint64_t* bufk = xbufk ? xbufk : (uint64_t*)(ws + lay.bufk);
    uint32_t* bufv = vals ? (xbufk ? xbufv : (uint32_t*)(ws + lay.bufv)) : nullptr;
    int64_t* rows = (int64_t*)(ws + lay.rows);
    uint8_t* levels = (uint8_t*)(ws + lay.levels);
    SegChunk* list = (SegChunk*)(ws + lay.list);
    const int64_t stride = nseg + 1;
    const int sms = num_sms_dev();
    cudaError_t e = cudaMemsetAsync(ctl, 0, 256, s);
    if (e != cudaSuccess) return e;
    e = launch(K_SEG_PLAN, ord_count_kernel, dim3((unsigned)ceil_div(nseg, 256)), dim3(256), 0, s, off, nseg, lay.L,
               rows, levels, skip, (const int*)ctl);
    if (e != cudaSuccess) return e;
    if (lay.L > 0) {
        e = launch(K_SEG_PLAN, seg_scan_kernel, dim3((unsigned)lay.L), dim3(1024), 0, s, rows, nseg, (const int*)ctl);
        if (e != cudaSuccess) return e;
    }
    e = launch(K_SEG_TILE, ord_tile_kernel<512, 16>, dim3((unsigned)ceil_div(n, ORD_T)), dim3(512),
               sizeof(SmemKV<8192>), s, keys, vals, bufk, bufv, n, off, nseg, (const uint8_t*)levels, skip, mode,
               (const int*)ctl);
    if (e != cudaSuccess) return e;
    for (int p = 0; p < lay.L; ++p) {
        const int64_t* prefix = rows + p * stride;
        e = launch(K_SEG_MERGE, ord_partition_kernel, dim3((unsigned)ceil_div(lay.max_items, 256)), dim3(256), 0, s,
                   (const uint64_t*)keys, (const uint64_t*)bufk, off, nseg, prefix, (const uint8_t*)levels, p, list,
                   (const int*)ctl);
        if (e != cudaSuccess) return e;
        const int64_t cap = (int64_t)sms * ws_ctas_per_sm<SEG_WS_STAGES>();
        const int64_t grid = lay.max_items < cap ? lay.max_items : cap;
        e = launch(K_SEG_MERGE, seg_merge_ws_kernel, dim3((unsigned)grid), dim3(WS_CONSUMERS + 32),
                   sizeof(WsSmemOut<WS_CHUNK, SEG_WS_STAGES>), s, keys, vals, bufk, bufv, n, (const SegChunk*)list,
                   (const int64_t*)(prefix + nseg), mode, call_err, wait_limit_ns(), (const int*)ctl);
        if (e != cudaSuccess) return e;
    }
    return publish_call_error(call_err, s);
}

// ---------------------------------------------------------------- tuning + graph cache
struct TuneEntry {
    int dev;
    int64_t n, nseg;
    const void* off;
    int sched;
};
struct GraphEntry {
    int dev;
    void *keys, *vals;
    const void* off;
    int64_t n, nseg;
    int mode, sched;
    cudaGraphExec_t exec;
    char* ws;
    uint64_t kernels;    // kernel launches inside the graph
};

std::mutex g_seg_mu;
std::vector<TuneEntry> g_tuned;
std::vector<GraphEntry> g_graphs;       // small LRU (most recent last)
constexpr size_t kMaxGraphs = 4;

cudaStream_t capture_stream()
{
    static std::vector<cudaStream_t> streams;
    int dev = 0;
    cudaGetDevice(&dev);
    if ((int)streams.size() <= dev) streams.resize(dev + 1, nullptr);
    if (!streams[dev]) cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    return streams[dev];
}

// Times every candidate schedule on a scratch copy of the input and returns the
// fastest (synchronises the stream).
int autotune(uint64_t* keys, uint32_t* vals, const int64_t* off, int64_t nseg, int64_t n, int mode,
             cudaStream_t s, int* rc)
{
    *rc = GNS_OK;
    const SegLayout lay = seg_layout(n, nseg, vals != nullptr);
    const size_t kb = align256((size_t)n * 8), vb = vals ? align256((size_t)n * 4) : 0;
    char* ws = (char*)ws_alloc(lay.total + 2 * (kb + vb), s);
    if (!ws) {
        *rc = GNS_ERR_OOM;
        return 0;
    }
    uint64_t* tk = (uint64_t*)(ws + lay.total);
    uint32_t* tv = vals ? (uint32_t*)(ws + lay.total + kb) : nullptr;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0;
    float best_ms = 1e30f;
    const int ncand = (int)(sizeof(kCandidates) / sizeof(kCandidates[0]));
    for (int c = 0; c < ncand && *rc == GNS_OK; ++c) {
        for (int rep = 0; rep < 2; ++rep) {   // first run warms up
            if (cudaMemcpyAsync(tk, keys, (size_t)n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                (vals && cudaMemcpyAsync(tv, vals, (size_t)n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)) {
                *rc = GNS_ERR_CUDA;
                break;
            }
            cudaEventRecord(e0, s);
            if (seg_enqueue(tk, tv, off, nseg, n, mode, kCandidates[c], ws, lay, s) != cudaSuccess) {
                *rc = GNS_ERR_CUDA;
                break;
            }
            cudaEventRecord(e1, s);
        }
        if (*rc != GNS_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ws_free(ws, s);
    return best;
}

}  // namespace

// Segmented sort entry (all checks done by the caller).
int segmented_sort_device(uint64_t* keys, uint32_t* vals, const int64_t* off, int64_t nseg, int64_t n, int mode,
                          cudaStream_t s)
{
    if (nseg == 0 || n <= 1) return GNS_OK;
    seg_init_attributes();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GNS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_seg_mu);
    // 1. the tuned schedule for this shape
    int sched = -1;
    for (auto& t : g_tuned)
        if (t.dev == dev && t.n == n && t.nseg == nseg && t.off == off) sched = t.sched;
    if (sched < 0) {
        const char* fixed = getenv("GNS_SEG_SCHEDULE");
        if (fixed) {
            sched = atoi(fixed);
            if (sched < 0 || sched >= (int)(sizeof(kCandidates) / sizeof(kCandidates[0]))) sched = 0;
        } else {
            int rc = GNS_OK;
            sched = autotune(keys, vals, off, nseg, n, mode, s, &rc);
            if (rc != GNS_OK) return rc;
        }
        g_tuned.push_back({dev, n, nseg, (const void*)off, sched});
    }
    // 2. the captured graph for these pointers
    for (size_t i = 0; i < g_graphs.size(); ++i) {
        GraphEntry& g = g_graphs[i];
        if (g.dev == dev && g.keys == keys && g.vals == vals && g.off == off && g.n == n && g.nseg == nseg &&
            g.mode == mode && g.sched == sched) {
            GraphEntry hit = g;
            g_graphs.erase(g_graphs.begin() + i);
            g_graphs.push_back(hit);
            g_launches.fetch_add(hit.kernels, std::memory_order_relaxed);
            return cudaGraphLaunch(hit.exec, s) == cudaSuccess ? GNS_OK : GNS_ERR_CUDA;
        }
    }
    const SegLayout lay = seg_layout(n, nseg, vals != nullptr);
    char* ws = (char*)ws_alloc(lay.total, s);
    if (!ws) return GNS_ERR_OOM;
    // the workspace must exist before the graph first runs
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        ws_free(ws, s);
        return GNS_ERR_CUDA;
    }
    if (!status_word_ptr()) {   // resolve the status word before capturing
        ws_free(ws, s);
        return GNS_ERR_CUDA;
    }
    cudaStream_t cs = capture_stream();
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    set_capturing(true);
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e2 = seg_enqueue(keys, vals, off, nseg, n, mode, kCandidates[sched], ws, lay, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (e2 != cudaSuccess) e = e2;
    }
    const uint64_t kernels = take_captured_launches();
    set_capturing(false);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ws_free(ws, s);
        return GNS_ERR_CUDA;
    }
    if (g_graphs.size() >= kMaxGraphs) {
        GraphEntry old = g_graphs.front();
        g_graphs.erase(g_graphs.begin());
        cudaStreamSynchronize(s);
        cudaGraphExecDestroy(old.exec);
        ws_free(old.ws, s);
    }
    g_graphs.push_back({dev, keys, vals, off, n, nseg, mode, sched, exec, ws, kernels});
    g_launches.fetch_add(kernels, std::memory_order_relaxed);
    return cudaGraphLaunch(exec, s) == cudaSuccess ? GNS_OK : GNS_ERR_CUDA;
}

size_t segmented_workspace_bytes(int64_t n, int64_t nseg, bool ext_buf)
{
    return seg_layout(n, nseg, true, ext_buf).total;
}

// Sort of ordered segments (see ord_count_kernel): the learned sort's buckets,
// built by the caller on the device.  off: nseg + 1 non-decreasing offsets
// with off[nseg] = n; skip (optional): segments known to be all tied; xbufk /
// xbufv (optional): a caller-provided n-element ping-pong buffer.  No tuning,
// no graph capture.  The segments must be ordered, which the bucket check
// after the call verifies.
int ordered_sort_direct(uint64_t* keys, uint32_t* vals, const int64_t* off, int64_t nseg, int64_t n, int mode,
                        const uint8_t* skip, cudaStream_t s, uint64_t* xbufk, uint32_t* xbufv)
{
    if (nseg == 0 || n <= 1) return GNS_OK;
    seg_init_attributes();
    const bool ext = xbufk != nullptr && (vals == nullptr || xbufv != nullptr);
    const SegLayout lay = seg_layout(n, nseg, vals != nullptr, ext);
    char* ws = (char*)ws_alloc(lay.total, s);
    if (!ws) return GNS_ERR_OOM;
    cudaError_t e = ord_enqueue(keys, vals, off, nseg, n, mode, ws, lay, s, skip, ext ? xbufk : nullptr,
                                ext ? xbufv : nullptr);
    ws_free(ws, s);
    return e == cudaSuccess ? GNS_OK : GNS_ERR_CUDA;
}

int segmented_schedule_of(int64_t n, int64_t nseg, const void* off)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_seg_mu);
    for (auto& t : g_tuned)
        if (t.dev == dev && t.n == n && t.nseg == nseg && t.off == off) return t.sched;
    return -1;
}

void segmented_release_graphs(cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_seg_mu);
    cudaStreamSynchronize(s);
    for (auto& g : g_graphs) {
        cudaGraphExecDestroy(g.exec);
        ws_free(g.ws, s);
    }
    g_graphs.clear();
    g_tuned.clear();
}

}  // namespace gns

using namespace gns;

extern "C" {

int gns_segmented_sort_ex(void* keys, int key_type, uint32_t* payload, const int64_t* offsets, int64_t nseg,
                          int64_t total_n, int order, gns_stream_t stream)
{
    if (nseg < 0 || total_n < 0) return GNS_ERR_INVALID;
    if (key_type != GNS_KEY_F64 && key_type != GNS_KEY_I64) return GNS_ERR_INVALID;
    if (order != GNS_ASCENDING && order != GNS_DESCENDING) return GNS_ERR_INVALID;
    if (nseg > 0 && offsets == nullptr) return GNS_ERR_INVALID;
    if (total_n > 0 && keys == nullptr) return GNS_ERR_INVALID;
    if (((uintptr_t)keys & 7) || ((uintptr_t)payload & 3) || ((uintptr_t)offsets & 7)) return GNS_ERR_INVALID;
    if (nseg > 0x7fffffff) return GNS_ERR_UNSUPPORTED;
    const int mode = (key_type == GNS_KEY_I64 ? MODE_I64 : 0) | (order == GNS_DESCENDING ? MODE_DESC : 0);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = segmented_sort_device((uint64_t*)keys, payload, offsets, nseg, total_n, mode, s);
    return finish_call(rc, s);
}

int gns_debug_ordered_segments(void* keys, int key_type, uint32_t* payload, int64_t n, const int64_t* offsets,
                               int64_t nseg, int order, gns_stream_t stream)
{
    if (nseg < 1 || n < 0 || offsets == nullptr) return GNS_ERR_INVALID;
    if (key_type != GNS_KEY_F64 && key_type != GNS_KEY_I64) return GNS_ERR_INVALID;
    if (order != GNS_ASCENDING && order != GNS_DESCENDING) return GNS_ERR_INVALID;
    if (n > 0 && keys == nullptr) return GNS_ERR_INVALID;
    if (((uintptr_t)keys & 7) || ((uintptr_t)payload & 3) || ((uintptr_t)offsets & 7)) return GNS_ERR_INVALID;
    if (nseg > 0x7fffffff) return GNS_ERR_UNSUPPORTED;
    const int mode = (key_type == GNS_KEY_I64 ? MODE_I64 : 0) | (order == GNS_DESCENDING ? MODE_DESC : 0);
    cudaStream_t s = (cudaStream_t)stream;
    const int rc = ordered_sort_direct((uint64_t*)keys, payload, offsets, nseg, n, mode, nullptr, s);
    return finish_call(rc, s);
}

int gns_segmented_sort(int64_t* keys, uint32_t* payload, const int64_t* offsets, int64_t nseg, gns_stream_t stream)
{
    if (nseg < 0) return GNS_ERR_INVALID;
    if (nseg == 0) return GNS_OK;
    if (offsets == nullptr) return GNS_ERR_INVALID;
    int64_t total = 0;
    // the host needs the total length to size the workspace: one 8-byte read
    if (cudaMemcpyAsync(&total, offsets + nseg, sizeof(int64_t), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
            cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return GNS_ERR_CUDA;
    return gns_segmented_sort_ex(keys, GNS_KEY_I64, payload, offsets, nseg, total, GNS_ASCENDING, stream);
}

int gns_segmented_schedule(int64_t total_n, int64_t nseg, const int64_t* offsets)
{
    return segmented_schedule_of(total_n, nseg, offsets);
}

void gns_segmented_release(gns_stream_t stream) { segmented_release_graphs((cudaStream_t)stream); }

}  // extern "C"
