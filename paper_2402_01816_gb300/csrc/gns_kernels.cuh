// gns_kernels.cuh -- the mergesort hot path on sm_103a.
//
//  tile sort        stable sort of a 4096-element tile in registers + shared memory:
//                   each thread sorts 16 keys with an odd-even transposition network
//                   (adjacent strict swaps only, hence stable), then 8 rounds of
//                   pairwise merges in shared memory, each thread finding its
//                   16-output slice by a merge-path co-rank search.
//  run detection    one read pass deciding "already in order" / "strictly reversed"
//                   (Omitsort / Octosort adaptivity, "Full adaptivity" section).
//  merge partition  merge-path co-rank of every CTA's first output, so that every
//                   merge level is split evenly over any number of CTAs (the
//                   "Parallel" section's binary merge over an arbitrary number of
//                   workers).
//  merge pass       one merge level: each CTA loads its two input slices to shared
//                   memory, merges 16 outputs per thread, stores coalesced.
//  frog kernels     the <= 50% buffer tier: the Frogsort1 layout ("Symmetric
//                   merging", "Frogsort1" sections) with a fused setup (tile sort +
//                   scatter to the gapped leaf slots) and in-place merge levels.
//
// All comparisons are on encoded keys (gns_device.cuh): one unsigned compare.
// Ties: the left run always wins, which makes every merge stable.
#pragma once

#include "gns_device.cuh"

namespace gns {

// Tile sort: SORT_THREADS x SORT_ITEMS elements per CTA (GNS_SORT_THREADS may
// be set at build time).
#ifndef GNS_SORT_THREADS
#define GNS_SORT_THREADS 512
#endif
constexpr int SORT_THREADS = GNS_SORT_THREADS;
constexpr int SORT_ITEMS = 16;
constexpr int TILE = SORT_THREADS * SORT_ITEMS;       // elements per tile (8192 by default)
// Merge levels work in chunks of CHUNK outputs, MERGE_ITEMS per consumer
// thread (gns_merge_ws.cuh); GNS_MERGE_CONSUMERS may be set at build time.
#ifndef GNS_MERGE_CONSUMERS
#define GNS_MERGE_CONSUMERS 256
#endif
constexpr int MERGE_CONSUMERS = GNS_MERGE_CONSUMERS;
#ifndef GNS_MERGE_ITEMS
#define GNS_MERGE_ITEMS 9
#endif
// 9 outputs per consumer thread: neighbouring lanes' run heads then lie 9
// elements (18 words) apart where a thread's outputs come from one run, and
// 4.5 apart where they alternate -- distinct banks either way.  With 8 (a
// 16-word stride) every lane's block starts at word 0 or 16 modulo 32 and
// such reads conflict 8-fold.  The last consumers of a chunk have nothing to do.
constexpr int MERGE_ITEMS = GNS_MERGE_ITEMS;
constexpr int CHUNK = MERGE_CONSUMERS == 128 ? 1024 : 2048;   // outputs per merge chunk
static_assert(MERGE_CONSUMERS * MERGE_ITEMS >= CHUNK, "merge chunk size");
constexpr int DETECT_TILE = 4096;

// Shared-memory index with one pad slot per 16 elements: thread t's blocked
// element j sits at 17 t + j, so a warp's blocked accesses hit distinct banks.
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

template <int N>
struct SmemKV {
    uint64_t k[N + N / 16 + 1];   // + 1: a serial merge may read the head one past its right run
    uint32_t v[N + N / 16];
};

// Number of A elements among the first `diag` outputs of the stable merge of
// A[0, na) and B[0, nb), left run winning ties.
template <typename GA, typename GB>
__device__ __forceinline__ int64_t merge_path(int64_t diag, int64_t na, int64_t nb, GA A, GB B)
{
    int64_t lo = imax64(0, diag - nb), hi = imin64(diag, na);
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (A(mid) <= B(diag - 1 - mid)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Serial stable merge of ITEMS outputs from shared-memory runs [i, ie) and
// [j, je) into registers; the runs must hold at least ITEMS elements between
// them.  The decision "take A" tests both bounds itself, so a run's head is
// reloaded without a bounds test: past the end of run A it reads run B's
// first element, past the end of run B at most one slot past the tile (the
// spare slot of SmemKV), and the value is never used.  The reload is one load
// from the taken element's successor, whichever run it is in (one load
// instruction per output instead of one per run).
template <int N, int ITEMS>
__device__ __forceinline__ void serial_merge(const SmemKV<N>& sm, int i, int ie, int j, int je,
                                             uint64_t (&k)[ITEMS], uint32_t (&v)[ITEMS])
{
    uint64_t ka = i < ie ? sm.k[pidx(i)] : ~0ull;
    uint64_t kb = j < je ? sm.k[pidx(j)] : ~0ull;
#pragma unroll
    for (int x = 0; x < ITEMS; ++x) {
        const bool takeA = (j >= je) || (i < ie && ka <= kb);
        const int src = takeA ? i : j;
        k[x] = takeA ? ka : kb;
        v[x] = sm.v[pidx(src)];
        const uint64_t next = sm.k[pidx(src + 1)];
        if (takeA) {
            ++i;
            ka = next;
        } else {
            ++j;
            kb = next;
        }
    }
}

// Stable sort of the tile held in shared memory at logical positions [0, T).
// Positions >= n_valid must hold the maximal key ~0 (they stay behind every
// real element: equal keys keep position order).  On return the sorted tile is
// at logical positions [0, n_valid) of `sm`.
template <int THREADS, int ITEMS>
__device__ void block_sort_smem(SmemKV<THREADS * ITEMS>& sm, int n_valid)
{
    constexpr int T = THREADS * ITEMS;
    const int t = threadIdx.x;
    uint64_t k[ITEMS];
    uint32_t v[ITEMS];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        k[j] = sm.k[pidx(t * ITEMS + j)];
        v[j] = sm.v[pidx(t * ITEMS + j)];
    }
    // odd-even transposition network: ITEMS phases of adjacent compare-swaps
#pragma unroll
    for (int ph = 0; ph < ITEMS; ++ph) {
#pragma unroll
        for (int j = ph & 1; j + 1 < ITEMS; j += 2) {
            if (k[j + 1] < k[j]) {
                uint64_t tk = k[j]; k[j] = k[j + 1]; k[j + 1] = tk;
                uint32_t tv = v[j]; v[j] = v[j + 1]; v[j + 1] = tv;
            }
        }
    }
    for (int w = ITEMS; w < T && w < n_valid; w <<= 1) {
        // while two runs span at most one warp's 32 * ITEMS positions, each
        // warp reads only what its own threads wrote: a warp barrier suffices
        const bool warp_local = 2 * w <= 32 * ITEMS;
        if (warp_local) __syncwarp(); else __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            sm.k[pidx(t * ITEMS + j)] = k[j];
            sm.v[pidx(t * ITEMS + j)] = v[j];
        }
        if (warp_local) __syncwarp(); else __syncthreads();
        const int gthreads = (2 * w) / ITEMS;
        const int a_beg = (t / gthreads) * 2 * w;
        const int b_beg = a_beg + w;
        const int diag = (t % gthreads) * ITEMS;
        // merge path in 32-bit indices (both runs hold w elements)
        int lo = diag - w > 0 ? diag - w : 0, hi = diag < w ? diag : w;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sm.k[pidx(a_beg + mid)] <= sm.k[pidx(b_beg + diag - 1 - mid)]) lo = mid + 1;
            else hi = mid;
        }
        serial_merge<T, ITEMS>(sm, a_beg + lo, b_beg, b_beg + diag - lo, b_beg + w, k, v);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        sm.k[pidx(t * ITEMS + j)] = k[j];
        sm.v[pidx(t * ITEMS + j)] = v[j];
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Run detection and reversal
// ---------------------------------------------------------------------------

// presorted[0]: every adjacent pair non-decreasing (under the call's order);
// presorted[1]: every adjacent pair strictly decreasing.  Both start at 1; any
// CTA finding a violation clears the flag.  Persistent CTAs walk tiles of
// DETECT_TILE keys (one coalesced load per key, staged in shared memory with the
// key before the tile) and stop as soon as both flags are cleared, so random
// inputs cost about one wave.
constexpr int DETECT_THREADS = 256;
static __global__ void __launch_bounds__(DETECT_THREADS) run_detect_kernel(const uint64_t* __restrict__ keys, int64_t n,
                                                         int mode, int* presorted)
{
    __shared__ uint64_t sk[DETECT_TILE + 1];
    __shared__ int s_go;
    const int t = threadIdx.x;
    for (int64_t tile = blockIdx.x; tile * DETECT_TILE < n; tile += gridDim.x) {
        if (t == 0) s_go = (ld_relaxed(&presorted[0]) | ld_relaxed(&presorted[1])) != 0;
        __syncthreads();
        if (!s_go) return;
        const int64_t base = tile * DETECT_TILE;
        const int cnt = (int)imin64(DETECT_TILE, n - base);     // pairs (g-1, g) for g in [base, base+cnt)
        // all of a thread's loads are issued before the first store (a loop that
        // stores each load before issuing the next serialises the latencies)
        constexpr int PER = DETECT_TILE / DETECT_THREADS + 1;
        uint64_t r[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int i = t + q * DETECT_THREADS;
            const int64_t g = base - 1 + i;
            r[q] = (i <= cnt && g >= 0) ? keys[g] : 0;
        }
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int i = t + q * DETECT_THREADS;
            if (i <= cnt) sk[i] = base - 1 + i >= 0 ? encode_key(r[q], mode) : 0;
        }
        __syncthreads();
        bool asc = true, desc = true;
        for (int i = t; i < cnt; i += blockDim.x) {
            if (base + i == 0) continue;
            uint64_t x = sk[i], y = sk[i + 1];
            asc &= (x <= y);
            desc &= (x > y);
        }
        asc = __syncthreads_and(asc);
        desc = __syncthreads_and(desc);
        if (t == 0) {   // clear a flag only while it is set: no atomic per tile on one word
            if (!asc && ld_relaxed(&presorted[0])) atomicAnd(&presorted[0], 0);
            if (!desc && ld_relaxed(&presorted[1])) atomicAnd(&presorted[1], 0);
        }
    }
}

// Reverses keys[0, n) and vals[0, n) in place (grid-stride over the CTAs).
__device__ __forceinline__ void reverse_body(uint64_t* keys, uint32_t* vals, int64_t n)
{
    const int64_t half = n / 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (n % 8 == 0 && ((uintptr_t)keys & 15) == 0 && ((uintptr_t)vals & 15) == 0) {
        // groups of four: group g = elements [4g, 4g + 4) and its mirror
        // [n - 4 - 4g, n - 4g), both 16-byte aligned, swapped with 16-byte accesses
        for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < half / 4; g += stride) {
            const int64_t i0 = 4 * g, j0 = n - 4 - 4 * g;
            ulonglong2* fk = reinterpret_cast<ulonglong2*>(keys + i0);
            ulonglong2* bk = reinterpret_cast<ulonglong2*>(keys + j0);
            uint4* fv = reinterpret_cast<uint4*>(vals + i0);
            uint4* bv = reinterpret_cast<uint4*>(vals + j0);
            // every load before the first store: one memory latency per group
            const ulonglong2 a01 = fk[0], a23 = fk[1], b01 = bk[0], b23 = bk[1];
            uint4 x = make_uint4(0, 0, 0, 0), y = x;
            if (vals) {
                x = *fv;
                y = *bv;
            }
            fk[0] = make_ulonglong2(b23.y, b23.x);
            fk[1] = make_ulonglong2(b01.y, b01.x);
            bk[0] = make_ulonglong2(a23.y, a23.x);
            bk[1] = make_ulonglong2(a01.y, a01.x);
            if (vals) {
                *fv = make_uint4(y.w, y.z, y.y, y.x);
                *bv = make_uint4(x.w, x.z, x.y, x.x);
            }
        }
        return;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < half; i += stride) {
        int64_t j = n - 1 - i;
        uint64_t a = keys[i], b = keys[j];
        keys[i] = b; keys[j] = a;
        if (vals) {
            uint32_t x = vals[i], y = vals[j];
            vals[i] = y; vals[j] = x;
        }
    }
}

// Reverses a strictly decreasing array in place (Octosort's final reversal: the
// reverse of a strictly ordered run is the stable sort, as it has no ties).
static __global__ void reverse_kernel(uint64_t* keys, uint32_t* vals, int64_t n, const int* presorted)
{
    if (presorted[0] != 0 || presorted[1] == 0) return;
    reverse_body(keys, vals, n);
}

// A sort whose start is decided on the device: with *gate == 0 the presorted
// flag is raised (every later kernel of the sort returns at once), otherwise
// both flags are cleared (no run detection: the sort runs in full).
static __global__ void gate_kernel(const int* gate, int* presorted)
{
    presorted[0] = (*gate == 0) ? 1 : 0;
    presorted[1] = 0;
}

// ctl[0..1]: presorted flags (nothing left to do), ctl[2]: the call's error
// word.  Every kernel after run detection returns at once when any is set, so
// that after a device-side error (a wait that ran out) no later pass runs on
// data the failed pass left half-written.
__device__ __forceinline__ bool skip_all(const int* ctl)
{
    return ctl != nullptr && (ctl[0] | ctl[1] | ld_relaxed(&ctl[2])) != 0;
}

// ---------------------------------------------------------------------------
// 100% tier: tile sort, partition, ping-pong merge pass
// ---------------------------------------------------------------------------

// Sorts tile blockIdx.x of src (raw keys) into dst (encoded keys, or raw when
// this is the only pass).  src == dst is allowed (each CTA owns its tile).
template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)   // <= 64 registers: 1024 threads per SM
    tile_sort_kernel(const uint64_t* src_k, const uint32_t* src_v, uint64_t* dst_k, uint32_t* dst_v,
                     int64_t n, int mode, int decode_out, const int* presorted)
{
    constexpr int T = THREADS * ITEMS;
    if (skip_all(presorted)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemKV<T>& sm = *reinterpret_cast<SmemKV<T>*>(smem_raw);
    const int t = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * T;
    const int nv = (int)imin64(T, n - base);
#pragma unroll 4
    for (int j = 0; j < ITEMS; ++j) {
        int i = t + j * THREADS;
        int64_t g = base + i;
        bool ok = i < nv;
        sm.k[pidx(i)] = ok ? encode_key(src_k[g], mode) : ~0ull;
        sm.v[pidx(i)] = (ok && src_v) ? src_v[g] : 0u;
    }
    block_sort_smem<THREADS, ITEMS>(sm, nv);
#pragma unroll 4
    for (int j = 0; j < ITEMS; ++j) {
        int i = t + j * THREADS;
        if (i < nv) {
            uint64_t key = sm.k[pidx(i)];
            dst_k[base + i] = decode_out ? decode_key(key, mode) : key;
            if (dst_v) dst_v[base + i] = sm.v[pidx(i)];
        }
    }
}

// splits[b] = co-rank (A elements) of output position b*CHUNK within its pair of
// runs of width w.
static __global__ void merge_partition_kernel(const uint64_t* __restrict__ k, int64_t n, int64_t w,
                                       int64_t nblocks, int64_t* splits, const int* presorted)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks || skip_all(presorted)) return;
    int64_t out0 = b * CHUNK;
    int64_t ps = (out0 / (2 * w)) * (2 * w);
    int64_t lenA = imin64(w, n - ps);
    int64_t lenB = imax64(0, imin64(w, n - ps - w));
    const uint64_t* A = k + ps;
    const uint64_t* B = k + ps + lenA;
    splits[b] = merge_path(out0 - ps, lenA, lenB, [&](int64_t x) { return A[x]; },
                           [&](int64_t x) { return B[x]; });
}

// ---------------------------------------------------------------------------
// <= 50% tier: the Frogsort1 layout
// ---------------------------------------------------------------------------
//
// A node sorts n elements inside a region of n + b slots starting at slot r; s is
// the input index of its first element.  side 0 = data-left (data ends in the
// region's left n slots), side 1 = data-right.  Left children are data-left,
// right children data-right, so the children's buffers meet in the middle of
// the parent's region.  The odd surplus element goes to the outer child (left
// child of a data-left node, right child of a data-right node); the root has
// b = floor(n/2); the outer child gets floor(n_outer/2) buffer slots, the inner
// child the rest -- never fewer than the inner child's element count, which is
// what the in-place merge needs.
//
// Slots [0, n) are the caller's arrays, slots [n, n + floor(n/2)) the buffer.
//
// ori is the orientation a node's sorted run is stored in (0 for every node of
// Frogsort1): 0 = ascending from left to right (the target order itself), 1 =
// its mirror image, the same sequence stored right to left.  The symmetric
// variants give nodes either orientation ("Symmetric merging" section:
// Geckosort sorts data-left branches left-ascending and data-right branches
// right-ascending; "Squidsort" section: the data decides, as in Octosort's
// lazily enforced order of the "Full adaptivity" section).  The in-place merge
// reads the outer child's run, which lies under the node's output, from its
// inner end, so a node always has its outer child's orientation; the inner
// child lies in the buffer and is read in whichever direction the node needs.

struct FrogNode {
    int64_t n, b, r, s;
    int32_t side, ori;
};

__host__ __device__ __forceinline__ void frog_split(const FrogNode& p, FrogNode& L, FrogNode& R)
{
    int64_t n_outer = (p.n + 1) / 2, n_inner = p.n - n_outer;
    int64_t b_outer = n_outer / 2, b_inner = p.b - b_outer;
    if (p.side == 0) { L.n = n_outer; L.b = b_outer; R.n = n_inner; R.b = b_inner; }
    else             { L.n = n_inner; L.b = b_inner; R.n = n_outer; R.b = b_outer; }
    L.side = 0; R.side = 1; L.ori = R.ori = 0;
    L.r = p.r; R.r = p.r + L.n + L.b;
    L.s = p.s; R.s = p.s + L.n;
}

__host__ __device__ __forceinline__ int64_t frog_data_slot(const FrogNode& x) { return x.side == 0 ? x.r : x.r + x.b; }

struct Slots {
    uint64_t* k0; uint32_t* v0;   // caller arrays: slots [0, n)
    uint64_t* k1; uint32_t* v1;   // buffer: slots [n, n + b)
    int64_t n;
    int64_t b;
    __device__ __forceinline__ uint64_t* kp(int64_t s) const { return s < n ? k0 + s : k1 + (s - n); }
    __device__ __forceinline__ uint32_t* vp(int64_t s) const { return s < n ? v0 + s : v1 + (s - n); }
};

// All nodes of depths 0..D in heap order: node k of depth d at (1 << d) - 1 + k.
// Each thread walks from the root down the bits of k.
static __global__ void frog_plan_kernel(FrogNode* nodes, int64_t n, int D)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = (2ll << D) - 1;
    if (idx >= total) return;
    int d = 63 - __clzll(idx + 1);
    int64_t k = idx + 1 - (1ll << d);
    FrogNode x;
    x.n = n; x.b = n / 2; x.r = 0; x.s = 0; x.side = 0; x.ori = 0;
    for (int lvl = d - 1; lvl >= 0; --lvl) {
        FrogNode L, R;
        frog_split(x, L, R);
        x = ((k >> lvl) & 1) ? R : L;
    }
    nodes[idx] = x;
}

// Largest leaf index j with leaves[j].s <= pos.
__device__ __forceinline__ int64_t find_leaf(const FrogNode* leaves, int64_t nleaves, int64_t pos)
{
    int64_t lo = 0, hi = nleaves - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (leaves[mid].s <= pos) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Leaf orientations of the symmetric variants (FrogNode::ori).
enum { FROG_PLAIN = 0, FROG_GECKO = 1, FROG_SQUID = 2 };

// Fused setup: every leaf's elements are read from the contiguous input, sorted
// as a tile and written to the leaf's gapped data slots (Frogsort1 setup; the
// destination is never left of the source).  A leaf's destination can overlap
// the input of leaves to its right, so leaves are processed in descending order
// by ticket, each publishes "inputs loaded" right after loading, and writes only
// once every overlapped leaf has published.  Earlier tickets never wait on later
// ones, so the waits cannot deadlock; they are bounded anyway.
//
// VARIANT picks the orientation each leaf's run is stored in (leaf_ori[leaf]
// receives it; unused for FROG_PLAIN):
//   FROG_PLAIN  ascending (Frogsort1);
//   FROG_GECKO  the leaf's side: data-left leaves ascending, data-right leaves
//               mirrored (Geckosort);
//   FROG_SQUID  decided by the data (Squidsort): mirrored when the leaf's input
//               is non-increasing and its first key lies strictly above its
//               last -- the leaf-sized form of Octosort's rule for two single
//               elements (mirrored when strictly out of order).
// A mirrored leaf stores its stable ascending sequence right to left; the
// result is the same stable sort whatever the orientations are.
template <int THREADS, int ITEMS, int VARIANT = FROG_PLAIN>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)   // <= 64 registers: 1024 threads per SM
    frog_setup_kernel(Slots sl, const FrogNode* __restrict__ leaves, int64_t nleaves, int mode,
                      int* ticket, int* loaded, int* call_err, uint64_t limit_ns,
                      const int* presorted, int* leaf_ori, uint32_t jitter_ns)
{
    constexpr int T = THREADS * ITEMS;
    if (skip_all(presorted)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemKV<T>& sm = *reinterpret_cast<SmemKV<T>*>(smem_raw);
    __shared__ int64_t s_leaf;
    __shared__ int s_ok;
    const int t = threadIdx.x;
    if (t == 0) {
        s_leaf = nleaves - 1 - atomicAdd(ticket, 1);
        debug_jitter(jitter_ns, s_leaf, 0);               // test hook: the leaf loads late
    }
    __syncthreads();
    const int64_t leaf = s_leaf;
    const FrogNode x = leaves[leaf];
    const int nv = (int)x.n;
#pragma unroll 4
    for (int j = 0; j < ITEMS; ++j) {
        int i = t + j * THREADS;
        bool ok = i < nv;
        int64_t g = x.s + i;
        sm.k[pidx(i)] = ok ? encode_key(sl.k0[g], mode) : ~0ull;
        sm.v[pidx(i)] = (ok && sl.v0) ? sl.v0[g] : 0u;
    }
    __syncthreads();
    if (t == 0) st_release(&loaded[leaf], 1);
    int ori = 0;
    if (VARIANT == FROG_GECKO) ori = x.side;
    if (VARIANT == FROG_SQUID) {
        bool nonincr = true;
        for (int i = t; i + 1 < nv; i += THREADS) nonincr &= sm.k[pidx(i)] >= sm.k[pidx(i + 1)];
        nonincr = __syncthreads_and(nonincr);
        ori = (nonincr && nv >= 2 && sm.k[pidx(0)] > sm.k[pidx(nv - 1)]) ? 1 : 0;
    }
    if (VARIANT != FROG_PLAIN && t == 0) leaf_ori[leaf] = ori;
    block_sort_smem<THREADS, ITEMS>(sm, nv);
    const int64_t dslot = frog_data_slot(x);
    if (t == 0) {
        bool ok = true;
        if (dslot < sl.n && nv > 0) {
            int64_t j0 = find_leaf(leaves, nleaves, dslot);
            int64_t j1 = find_leaf(leaves, nleaves, imin64(dslot + nv - 1, sl.n - 1));
            for (int64_t j = imax64(j0, leaf + 1); j <= j1 && ok; ++j)
                ok = wait_flag(&loaded[j], 1, call_err, limit_ns, GNS_ERR_TIMEOUT);
        }
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
#pragma unroll 4
    for (int j = 0; j < ITEMS; ++j) {
        int i = t + j * THREADS;
        if (i < nv) {
            const int64_t d = dslot + (ori ? nv - 1 - i : i);
            *sl.kp(d) = sm.k[pidx(i)];
            if (sl.v0) *sl.vp(d) = sm.v[pidx(i)];
        }
    }
}

// Orientation of every node of the Frogsort1 tree (heap order, depths 0..D)
// from its leaves' (symmetric variants): a node takes its outer child's
// orientation, and the outer child of a data-left node is its left child,
// which is data-left again, so a data-left node has its leftmost leaf's
// orientation and a data-right node its rightmost leaf's.
static __global__ void frog_orient_kernel(FrogNode* nodes, int D, const int* __restrict__ leaf_ori,
                                          const int* presorted)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (2ll << D) - 1 || skip_all(presorted)) return;
    const int d = 63 - __clzll(idx + 1);
    const int64_t k = idx + 1 - (1ll << d);
    const int sh = D - d;
    const int64_t leaf = nodes[idx].side == 0 ? (k << sh) : ((k + 1) << sh) - 1;
    nodes[idx].ori = leaf_ori[leaf];
}

// The chunks of a level's nodes are numbered node by node: node k's chunks
// are [cstart[k], cstart[k+1]).  cstart == nullptr: every node has nch chunk
// slots (the balanced Frogsort1 tree; slots past a node's end are empty).
__device__ __forceinline__ void frog_locate(int64_t idx, const int64_t* __restrict__ cstart, int64_t nnodes,
                                            int64_t nch, int64_t& k, int64_t& local, int64_t& base, int64_t& nchk)
{
    if (!cstart) {
        k = idx / nch;
        local = idx % nch;
        base = k * nch;
        nchk = nch;
        return;
    }
    int64_t lo = 0, hi = nnodes - 1;                 // last k with cstart[k] <= idx
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (cstart[mid] <= idx) lo = mid;
        else hi = mid - 1;
    }
    k = lo;
    base = cstart[k];
    local = idx - base;
    nchk = cstart[k + 1] - base;
}

// frog_orient_kernel for a tree planned on the host (Frogsort2): node i of the
// list takes the orientation of leaf outer_leaf[i], its outermost leaf.
static __global__ void frog_orient_list_kernel(FrogNode* nodes, int64_t count, const int32_t* __restrict__ outer_leaf,
                                               const int* __restrict__ leaf_ori, const int* presorted)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count || skip_all(presorted)) return;
    nodes[i].ori = leaf_ori[outer_leaf[i]];
}

// splits[base(k) + c] = co-rank (left-run elements) of output c*CHUNK of node k.
//
// SYM (nodes of either orientation): the merge runs in slot order.  An
// ascending node takes its left run first on ties; a mirrored node stores the
// sequence right to left, so in slot order its larger keys come first and, of
// equal keys, the later one (the right run's).  So the first run F is the
// left child of an ascending node and the right child of a mirrored one, keys
// are compared after XOR with the node's mask (all ones when mirrored), F wins
// ties, and a child whose orientation differs from the node's is read from its
// far end.  splits then count F's elements.
template <bool SYM>
__global__ void frog_partition_kernel(Slots sl, const FrogNode* __restrict__ level,
                                      const FrogNode* __restrict__ child, int64_t nnodes, int64_t nch,
                                      const int64_t* __restrict__ cstart, int64_t total, int64_t* splits,
                                      const int* presorted)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total || skip_all(presorted)) return;
    int64_t k, c, base, nchk;
    frog_locate(idx, cstart, nnodes, nch, k, c, base, nchk);
    FrogNode x = level[k], L = child[2 * k], R = child[2 * k + 1];
    int64_t diag = imin64(c * CHUNK, x.n);
    if (!SYM) {
        int64_t ra = frog_data_slot(L), rb = frog_data_slot(R);
        splits[idx] = merge_path(diag, L.n, R.n, [&](int64_t i) { return *sl.kp(ra + i); },
                                 [&](int64_t j) { return *sl.kp(rb + j); });
        return;
    }
    const bool desc = x.ori != 0;
    const FrogNode F = desc ? R : L, S = desc ? L : R;
    const uint64_t mask = desc ? ~0ull : 0ull;
    const int64_t fd = frog_data_slot(F), sd = frog_data_slot(S);
    const bool rf = F.ori != x.ori, rs = S.ori != x.ori;
    splits[idx] = merge_path(
        diag, F.n, S.n, [&](int64_t i) { return *sl.kp(rf ? fd + F.n - 1 - i : fd + i) ^ mask; },
        [&](int64_t j) { return *sl.kp(rs ? sd + S.n - 1 - j : sd + j) ^ mask; });
}

// Squidsort's one final reversal: a root stored mirrored is reversed in place
// after its last level (the root is data-left: slots [0, n)).  Skipped when the
// whole sort was (presorted or reversed input, or an error).
static __global__ void reverse_root_kernel(uint64_t* keys, uint32_t* vals, int64_t n, const FrogNode* root,
                                           const int* ctl)
{
    if (skip_all(ctl) || root->ori == 0) return;
    reverse_body(keys, vals, n);
}

// One in-place symmetric merge level (kernel: frog_merge_tma_kernel).  A
// data-left node writes its output to slots [r, r+n); the only inputs it can
// overwrite are its left run's elements (they move right), so its chunks run
// from the top down (descending tickets) and chunk c writes after every later
// chunk that reads the left-run elements under it has loaded.  A data-right
// node (output [r+b, r+b+n)) is the mirror image: its right run's elements move
// left, chunks run bottom up.  The right (left) run of a data-left (data-right)
// node is never overwritten, because the node holds at least as many buffer
// slots as its inner child has elements.

static __global__ void publish_err_kernel(const int* call_err, int* status)
{
    int e = *call_err;
    if (e != 0) atomicCAS(status, 0, e);
}

}  // namespace gns
