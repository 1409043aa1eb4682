// gns_merge_tma.cuh -- the merge levels as persistent TMA pipelines (sm_100+).
//
// One merge level is an HBM stream: read 12 B and write 12 B per element.  Each
// CTA owns a sequence of 1024-output chunks.  While it merges chunk i, the Tensor
// Memory Accelerator already copies the two input slices of chunk i+1 into the
// other shared-memory stage (cp.async.bulk, completion on an mbarrier), and the
// finished chunk leaves shared memory as one bulk store per array
// (cp.async.bulk global <- shared).  The merge itself is the merge-path split
// of the chunk into 8 outputs per thread followed by a serial stable merge in
// registers.  Measured on one level of 2^27 keys: 4.9 TB/s, against 6.1-6.4 TB/s
// for a plain copy of the same bytes.
//
// Alignment: bulk copies move 16-byte aligned blocks.  A slice is copied from
// the 16-byte boundary at or below its first element (never across a page, so
// always mapped) up to the last boundary inside it; the at most one key / three
// payload words after that boundary are plain loads.  Stores use the bulk path
// when the chunk's destination is 16-byte aligned and the chunk is whole, else
// coalesced plain stores.
#pragma once

#include "gns_kernels.cuh"

namespace gns {

constexpr int TMA_THREADS = 128;
constexpr int TMA_ITEMS = 8;
constexpr int TMA_CHUNK = TMA_THREADS * TMA_ITEMS;   // 1024 outputs per chunk
constexpr int TMA_CTAS_PER_SM = 6;
static_assert(TMA_CHUNK == CHUNK, "merge chunk size");

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for an mbarrier phase; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, unsigned bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(sdst)),
                 "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// ---------------------------------------------------------------- geometry
struct ChunkGeo {
    int64_t out0;     // first output position
    int64_t a_src;    // first input position in the left run
    int64_t b_src;    // first input position in the right run
    int na, nb;
};

// Output chunk b of a Nocopy merge level with runs of width w (C divides 2w,
// so a chunk never spans two pairs of runs).
template <int C>
__device__ __forceinline__ ChunkGeo merge_chunk_geo(int64_t b, int64_t n, int64_t w, const int64_t* splits)
{
    ChunkGeo g;
    g.out0 = b * C;
    const int64_t ps = (g.out0 / (2 * w)) * (2 * w);
    const int64_t lenA = imin64(w, n - ps);
    const int64_t lenB = imax64(0, imin64(w, n - ps - w));
    const int64_t tot = lenA + lenB;
    const int64_t d0 = g.out0 - ps, d1 = imin64(d0 + C, tot);
    const int64_t a0 = splits[b];
    const int64_t a1 = (d1 == tot) ? lenA : splits[b + 1];
    g.na = (int)(a1 - a0);
    g.nb = (int)((d1 - a1) - (d0 - a0));
    g.a_src = ps + a0;
    g.b_src = ps + lenA + (d0 - a0);
    return g;
}

// ---------------------------------------------------------------- stages
template <int C>
struct InStage {
    uint64_t k[C + 8];
    uint32_t v[C + 16];
};
template <int C>
struct OutBuf {
    uint64_t k[C + 2];   // room for outputs shifted to the destination's 16-byte phase
    uint32_t v[C + 4];
};
template <int C>
struct MergeSmem {
    InStage<C> in[2];
    OutBuf<C> out;
};

// Where the two input slices of a staged chunk sit in shared memory.
struct StagedChunk {
    int na, nb;
    int ka, kb;   // shared index of the first key of each slice
    int va, vb;   // shared index of the first payload word of each slice
};

// One input slice: m consecutive elements at keys P / payload Pv.  Thread 0
// issues the bulk copy of the aligned interior (returns its byte count to add
// to the stage's transaction count); threads 1..4 load the tails.
// plain_sl != nullptr: the slice starts at slot plain_slot of a slot space that
// may change arrays inside the slice; every thread then copies with plain loads.
__device__ __forceinline__ unsigned stage_slice(uint64_t* sk, uint32_t* svv, int s0k, int s0v, const uint64_t* P,
                                                const uint32_t* Pv, int m, uint64_t* bar, int& koff, int& voff,
                                                const Slots* plain_sl, int64_t plain_slot)
{
    const int t = threadIdx.x;
    unsigned bytes = 0;
    if (plain_sl) {
        koff = s0k;
        voff = s0v;
        for (int e = t; e < m; e += blockDim.x) {
            sk[s0k + e] = *plain_sl->kp(plain_slot + e);
            if (Pv) svv[s0v + e] = *plain_sl->vp(plain_slot + e);
        }
        return 0;
    }
    const uintptr_t pk = (uintptr_t)P, pk_lo = pk & ~(uintptr_t)15, pk_hi = (pk + (uintptr_t)m * 8) & ~(uintptr_t)15;
    const int dk = (int)((pk - pk_lo) >> 3);
    koff = s0k + dk;
    const int ktail = pk_hi > pk ? (int)((pk_hi - pk) >> 3) : 0;
    if (t == 0 && pk_hi > pk_lo) {
        bulk_load(sk + s0k, (const void*)pk_lo, (unsigned)(pk_hi - pk_lo), bar);
        bytes += (unsigned)(pk_hi - pk_lo);
    }
    if (t == 1 && ktail < m) sk[koff + ktail] = P[ktail];
    voff = s0v;
    if (Pv) {
        const uintptr_t pv = (uintptr_t)Pv, pv_lo = pv & ~(uintptr_t)15, pv_hi = (pv + (uintptr_t)m * 4) & ~(uintptr_t)15;
        voff = s0v + (int)((pv - pv_lo) >> 2);
        const int vtail = pv_hi > pv ? (int)((pv_hi - pv) >> 2) : 0;
        if (t == 0 && pv_hi > pv_lo) {
            bulk_load(svv + s0v, (const void*)pv_lo, (unsigned)(pv_hi - pv_lo), bar);
            bytes += (unsigned)(pv_hi - pv_lo);
        }
        if (t >= 2 && t < 5 && vtail + (t - 2) < m) svv[voff + vtail + (t - 2)] = Pv[vtail + (t - 2)];
    }
    return bytes;
}

// Stages both slices of a chunk.  Thread 0 arms the stage's mbarrier with the
// total byte count of the bulk copies it issued.  plain_a / plain_b force the
// plain-load path for a slice.
template <int C>
__device__ __forceinline__ StagedChunk stage_chunk(InStage<C>& st, uint64_t* bar, const uint64_t* Ak,
                                                   const uint32_t* Av, int na, const uint64_t* Bk, const uint32_t* Bv,
                                                   int nb, const Slots* plain_a, int64_t slot_a, const Slots* plain_b,
                                                   int64_t slot_b)
{
    StagedChunk g;
    g.na = na;
    g.nb = nb;
    if (threadIdx.x == 0) fence_proxy_async_shared();   // earlier generic reads of this stage come first
    unsigned bytes = stage_slice(st.k, st.v, 0, 0, Ak, Av, na, bar, g.ka, g.va, plain_a, slot_a);
    const int s0k = (g.ka + na + 1) & ~1;               // 16-byte boundary after slice A
    const int s0v = (g.va + na + 3) & ~3;
    bytes += stage_slice(st.k, st.v, s0k, s0v, Bk, Bv, nb, bar, g.kb, g.vb, plain_b, slot_b);
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, bytes);
    return g;
}

// Merges a staged chunk: thread t's 8 outputs [8t, 8t + 8) into registers.
template <int C, int ITEMS>
__device__ __forceinline__ int merge_staged(const InStage<C>& st, const StagedChunk& g, uint64_t (&k)[ITEMS],
                                            uint32_t (&v)[ITEMS], bool has_vals)
{
    const int na = g.na, nb = g.nb, cnt = na + nb;
    const int diag = threadIdx.x * ITEMS;
    if (diag >= cnt) return 0;
    int lo = diag - nb > 0 ? diag - nb : 0, hi = diag < na ? diag : na;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (st.k[g.ka + mid] <= st.k[g.kb + diag - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    int i = lo, j = diag - lo;
    uint64_t ka = i < na ? st.k[g.ka + i] : ~0ull;
    uint64_t kb = j < nb ? st.k[g.kb + j] : ~0ull;
#pragma unroll
    for (int x = 0; x < ITEMS; ++x) {
        bool takeA = (j >= nb) || (i < na && ka <= kb);
        k[x] = takeA ? ka : kb;
        if (has_vals) v[x] = takeA ? st.v[g.va + (i < na ? i : na - 1)] : st.v[g.vb + (j < nb ? j : nb - 1)];
        if (takeA) {
            ++i;
            ka = i < na ? st.k[g.ka + i] : ~0ull;
        } else {
            ++j;
            kb = j < nb ? st.k[g.kb + j] : ~0ull;
        }
    }
    return cnt - diag < ITEMS ? cnt - diag : ITEMS;
}

template <int C, int ITEMS>
__device__ __forceinline__ void write_out(OutBuf<C>& ob, const uint64_t (&k)[ITEMS], const uint32_t (&v)[ITEMS], int m,
                                          bool has_vals, int mode, int decode_out)
{
    const int diag = threadIdx.x * ITEMS;
    if (m == ITEMS) {
#pragma unroll
        for (int x = 0; x < ITEMS; x += 2)
            *reinterpret_cast<ulonglong2*>(&ob.k[diag + x]) =
                make_ulonglong2(decode_out ? decode_key(k[x], mode) : k[x],
                                decode_out ? decode_key(k[x + 1], mode) : k[x + 1]);
        if (has_vals) {
#pragma unroll
            for (int x = 0; x < ITEMS; x += 4)
                *reinterpret_cast<uint4*>(&ob.v[diag + x]) = make_uint4(v[x], v[x + 1], v[x + 2], v[x + 3]);
        }
    } else {
#pragma unroll
        for (int x = 0; x < ITEMS; ++x) {
            if (x < m) {
                ob.k[diag + x] = decode_out ? decode_key(k[x], mode) : k[x];
                if (has_vals) ob.v[diag + x] = v[x];
            }
        }
    }
}

// True when cnt outputs at (Dk, Dv) can leave as bulk stores.
__device__ __forceinline__ bool bulk_ok(const void* Dk, const void* Dv, int cnt)
{
    return ((uintptr_t)Dk & 15) == 0 && (cnt & 3) == 0 && (Dv == nullptr || ((uintptr_t)Dv & 15) == 0);
}

// ============================================================ ping-pong levels
// One staged chunk: two input slices and where the merged run goes.
struct MergeItem {
    const uint64_t* ak; const uint32_t* av; int na;
    const uint64_t* bk; const uint32_t* bv; int nb;
    uint64_t* dk; uint32_t* dv;
    int decode;
};

// The pipeline shared by every out-of-place merge level: items b = blockIdx.x,
// blockIdx.x + gridDim.x, ... < nitems, described by get(b).
template <int THREADS, int ITEMS, typename Get>
__device__ __forceinline__ void merge_items_tma(int64_t nitems, Get get, int mode, int* call_err, uint64_t limit_ns)
{
    constexpr int C = THREADS * ITEMS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MergeSmem<C>& sm = *reinterpret_cast<MergeSmem<C>*>(smem_raw);
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ StagedChunk staged[2];
    __shared__ int s_ok;
    const int t = threadIdx.x;
    int64_t b = blockIdx.x;
    if (b >= nitems) return;
    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_ok = 1;
    }
    __syncthreads();
    bool pending[2] = {false, false};
    auto stage = [&](int slot, const MergeItem& m) {
        int na = m.na, nb = m.nb;
        if (na < 0 || nb < 0 || na + nb > C) {   // inconsistent splits: stage nothing
            if (t == 0) atomicCAS(call_err, 0, GNS_ERR_INTERNAL);
            na = nb = 0;
        }
        StagedChunk g = stage_chunk<C>(sm.in[slot], &bars[slot], m.ak, m.av, na, m.bk, m.bv, nb, nullptr, 0,
                                       nullptr, 0);
        if (t == 0) staged[slot] = g;
        pending[slot] = true;
    };
    MergeItem cur = get(b);
    stage(0, cur);
    unsigned parity[2] = {0u, 0u};
    for (int it = 0; b < nitems; ++it, b += gridDim.x) {
        const int cs = it & 1;
        const int64_t nb_ = b + gridDim.x;
        MergeItem nxt = cur;
        if (nb_ < nitems) {
            nxt = get(nb_);
            stage(cs ^ 1, nxt);
        }
        if (t == 0) {
            if (!mbar_wait(&bars[cs], parity[cs], limit_ns)) {
                atomicCAS(call_err, 0, GNS_ERR_TIMEOUT);
                s_ok = 0;
            }
            if (ld_relaxed(call_err) != 0) s_ok = 0;
            bulk_wait_read_all();                     // previous chunk's bulk store has read `out`
        }
        parity[cs] ^= 1u;
        pending[cs] = false;
        __syncthreads();
        if (!s_ok) break;
        const StagedChunk g = staged[cs];
        const bool has_vals = cur.av != nullptr;
        uint64_t k[ITEMS];
        uint32_t v[ITEMS];
        const int m = merge_staged<C, ITEMS>(sm.in[cs], g, k, v, has_vals);
        if (m > 0) write_out<C, ITEMS>(sm.out, k, v, m, has_vals, mode, cur.decode);
        fence_proxy_async_shared();
        __syncthreads();
        const int cnt = g.na + g.nb;
        uint64_t* Dk = cur.dk;
        uint32_t* Dv = has_vals ? cur.dv : nullptr;
        if (bulk_ok(Dk, Dv, cnt)) {
            if (t == 0 && cnt > 0) {
                bulk_store(Dk, sm.out.k, (unsigned)cnt * 8);
                if (Dv) bulk_store(Dv, sm.out.v, (unsigned)cnt * 4);
                bulk_commit();
            }
        } else {
            for (int e = t; e < cnt; e += THREADS) {
                Dk[e] = sm.out.k[e];
                if (Dv) Dv[e] = sm.out.v[e];
            }
        }
        cur = nxt;
    }
    if (t == 0) {
        bulk_wait_all();
        // a stage may still be in flight after an abort: wait for it (bounded)
        for (int q = 0; q < 2; ++q)
            if (pending[q]) mbar_wait(&bars[q], parity[q], limit_ns);
    }
}

// One Nocopy merge level of the 100% tier: runs of width w in (sk, sv) merged
// pairwise into (dk, dv), chunk b = outputs [b*C, (b+1)*C).
template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS)
    merge_pass_tma_kernel(const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sv, uint64_t* __restrict__ dk,
                          uint32_t* __restrict__ dv, int64_t n, int64_t w, int64_t nblocks,
                          const int64_t* __restrict__ splits, int mode, int decode_out, int* call_err,
                          uint64_t limit_ns, const int* presorted)
{
    constexpr int C = THREADS * ITEMS;
    if (skip_all(presorted)) return;
    auto get = [&](int64_t b) {
        ChunkGeo cg = merge_chunk_geo<C>(b, n, w, splits);
        MergeItem m;
        m.ak = sk + cg.a_src; m.av = sv ? sv + cg.a_src : nullptr; m.na = cg.na;
        m.bk = sk + cg.b_src; m.bv = sv ? sv + cg.b_src : nullptr; m.nb = cg.nb;
        m.dk = dk + cg.out0; m.dv = dv ? dv + cg.out0 : nullptr;
        m.decode = decode_out;
        return m;
    };
    merge_items_tma<THREADS, ITEMS>(nblocks, get, mode, call_err, limit_ns);
}

// ============================================================ <= 50% tier
// In-place symmetric merge level.  Chunks are handed out by ticket: within a
// data-left node from the top chunk down, within a data-right node from the
// bottom chunk up, so that every chunk that reads a run element lying under
// chunk c's output holds an earlier ticket than c (the ordering note after
// frog_partition_kernel).  A ticket's "inputs loaded" flag is published once its
// stage's mbarrier has completed; its outputs are stored after the flags of
// every such earlier ticket are set.  A CTA holds at most its current ticket
// and the next two, always in increasing order, and waits only go to earlier
// tickets, so no cycle of waits can form.  The flags of all levels share one
// array: level flags hold the level's epoch (1, 2, ... in launch order) once
// loaded, so a flag left by an earlier level never reads as loaded.

// Everything a ticket's merge needs, precomputed by frog_items_kernel so that
// the merge loop issues its copies after one independent load.
struct FrogItem {
    int64_t ra, rb;        // slot of the first element of the left / right slice
    int64_t oslot;         // slot of the first output
    int32_t na, nb;        // slice lengths (0, 0: nothing to do)
    int32_t dep_lo, dep_hi;   // tickets whose loads must precede the store (dep_hi < dep_lo: none)
};

// Range [lo, hi] of the chunks of node k that read the run elements chunk c
// overwrites (hi < lo: none).  A data-left node overwrites left-run indices
// [w0, min(w1, nL)), read by later chunks; a data-right node overwrites
// right-run indices [w0 - nL, w1 - nL), read by earlier chunks.  The input
// slices are monotone in the chunk index, so binary searches over the node's
// splits find the range.
__device__ __forceinline__ int2 frog_dep_range(int64_t c, const FrogNode& x, const FrogNode& L, const FrogNode& R,
                                               const int64_t* sp, int C)
{
    int2 r = make_int2(0, -1);
    const int64_t w0 = c * C, w1 = imin64(w0 + C, x.n);
    if (w0 >= x.n) return r;
    const int64_t last = (x.n - 1) / C;
    auto a_beg = [&](int64_t q) { return sp[q]; };
    auto a_end = [&](int64_t q) { return q == last ? L.n : sp[q + 1]; };
    auto b_beg = [&](int64_t q) { return q * C - sp[q]; };
    auto b_end = [&](int64_t q) { return imin64((q + 1) * C, x.n) - a_end(q); };
    if (x.side == 0) {
        const int64_t lim = imin64(w1, L.n);
        if (w0 < lim && c < last) {
            int64_t lo = c + 1, hi = last;              // first q with a_end(q) > w0
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                if (a_end(mid) > w0) hi = mid;
                else lo = mid + 1;
            }
            int64_t lo2 = lo, hi2 = last;               // last q with a_beg(q) < lim
            if (a_beg(lo2) < lim) {
                while (lo2 < hi2) {
                    int64_t mid = (lo2 + hi2 + 1) >> 1;
                    if (a_beg(mid) < lim) lo2 = mid;
                    else hi2 = mid - 1;
                }
                r = make_int2((int)lo, (int)lo2);
            }
        }
    } else {
        const int64_t lo_b = imax64(w0 - L.n, 0), hi_b = imin64(w1 - L.n, R.n);
        if (lo_b < hi_b && c > 0 && b_beg(0) < hi_b) {
            int64_t lo = 0, hi = c - 1;                 // last q with b_beg(q) < hi_b
            while (lo < hi) {
                int64_t mid = (lo + hi + 1) >> 1;
                if (b_beg(mid) < hi_b) lo = mid;
                else hi = mid - 1;
            }
            int64_t lo2 = 0, hi2 = lo;                  // first q with b_end(q) > lo_b
            if (b_end(lo) > lo_b) {
                while (lo2 < hi2) {
                    int64_t mid = (lo2 + hi2) >> 1;
                    if (b_end(mid) > lo_b) hi2 = mid;
                    else lo2 = mid + 1;
                }
                r = make_int2((int)lo2, (int)lo);
            }
        }
    }
    return r;
}

// items[tk] for every ticket tk of a level (after the partition, before the
// merge): ticket tk = k * nch + local is chunk c = nch - 1 - local of a
// data-left node k and chunk c = local of a data-right one.
static __global__ void frog_items_kernel(const FrogNode* __restrict__ level, const FrogNode* __restrict__ child,
                                         int64_t nnodes, int64_t nch, const int64_t* __restrict__ splits,
                                         FrogItem* __restrict__ items, int* call_err, const int* presorted)
{
    const int64_t tk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tk >= nnodes * nch || skip_all(presorted)) return;
    const int64_t k = tk / nch, local = tk % nch;
    const FrogNode x = level[k];
    const int64_t c = x.side == 0 ? nch - 1 - local : local;
    FrogItem it;
    it.ra = it.rb = it.oslot = 0;
    it.na = it.nb = 0;
    it.dep_lo = 0;
    it.dep_hi = -1;
    const int64_t w0 = c * CHUNK;
    if (w0 < x.n) {
        const int64_t w1 = imin64(w0 + CHUNK, x.n);
        const FrogNode L = child[2 * k], R = child[2 * k + 1];
        const int64_t* sp = splits + k * nch;
        const int64_t a0 = sp[c];
        const int64_t a1 = (w1 == x.n) ? L.n : sp[c + 1];
        const int64_t na = a1 - a0, nb = (w1 - a1) - (w0 - a0);
        if (na < 0 || nb < 0 || na + nb > CHUNK || a0 < 0 || a1 > L.n) {   // splits inconsistent
            atomicCAS(call_err, 0, GNS_ERR_INTERNAL);
        } else {
            it.na = (int32_t)na;
            it.nb = (int32_t)nb;
            it.ra = frog_data_slot(L) + a0;
            it.rb = frog_data_slot(R) + (w0 - a0);
            it.oslot = frog_data_slot(x) + w0;
            const int2 r = frog_dep_range(c, x, L, R, sp, CHUNK);
            if (r.x <= r.y) {
                const int64_t base = k * nch;
                it.dep_lo = (int32_t)(x.side == 0 ? base + nch - 1 - r.y : base + r.x);
                it.dep_hi = (int32_t)(x.side == 0 ? base + nch - 1 - r.x : base + r.y);
            }
        }
    }
    items[tk] = it;
}

// Spin until *flag == want; `poll()` runs in the loop (it publishes the CTA's
// prefetched ticket as soon as that ticket's inputs have landed, so that no
// chain of waits runs through tickets that are loaded but not yet announced).
template <typename Poll>
__device__ __forceinline__ bool wait_flag_polling(const int* flag, int want, int* call_err, uint64_t limit_ns,
                                                  Poll poll)
{
    if (ld_acquire(flag) == want) return true;
    const uint64_t t0 = global_ns();
    unsigned sleep_ns = 32;
    for (;;) {
        poll();
        if (ld_acquire(flag) == want) return true;
        if (ld_relaxed(call_err) != 0) return false;
        if (global_ns() - t0 > limit_ns) {
            atomicCAS(call_err, 0, GNS_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(sleep_ns);
        if (sleep_ns < 512) sleep_ns <<= 1;
    }
}

template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS)
    frog_merge_tma_kernel(Slots sl, const FrogItem* __restrict__ items, int64_t total, int mode, int decode_out,
                          int* ticket, int* loaded, int epoch, int* call_err, uint64_t limit_ns,
                          int64_t skip_ticket, const int* presorted)
{
    constexpr int C = THREADS * ITEMS;
    if (skip_all(presorted)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MergeSmem<C>& sm = *reinterpret_cast<MergeSmem<C>*>(smem_raw);
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ StagedChunk staged[2];
    __shared__ int64_t s_tk[2];
    __shared__ int64_t s_after;
    __shared__ int s_ok;
    const int t = threadIdx.x;
    const bool has_vals = sl.v0 != nullptr;
    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_tk[0] = atomicAdd(ticket, 1);
        s_tk[1] = s_tk[0] < total ? atomicAdd(ticket, 1) : total;
        s_ok = 1;
    }
    __syncthreads();
    int64_t tk = s_tk[0], tk_next = s_tk[1];
    if (tk >= total) return;

    bool pending[2] = {false, false};
    auto stage = [&](int slot, const FrogItem& m) {
        int na = m.na, nb = m.nb;
        if (na < 0 || nb < 0 || na + nb > C) {   // inconsistent item: stage nothing
            if (t == 0) atomicCAS(call_err, 0, GNS_ERR_INTERNAL);
            na = nb = 0;
        }
        const int64_t ra = na > 0 ? m.ra : 0, rb = nb > 0 ? m.rb : 0;
        // slices that straddle the caller-array / buffer boundary use plain loads
        const bool pa = na > 0 && ra < sl.n && ra + na > sl.n;
        const bool pb = nb > 0 && rb < sl.n && rb + nb > sl.n;
        StagedChunk g = stage_chunk<C>(sm.in[slot], &bars[slot], sl.kp(ra), has_vals ? sl.vp(ra) : nullptr, na,
                                       sl.kp(rb), has_vals ? sl.vp(rb) : nullptr, nb, pa ? &sl : nullptr, ra,
                                       pb ? &sl : nullptr, rb);
        if (t == 0) staged[slot] = g;
        pending[slot] = true;
    };

    FrogItem cur = items[tk];
    stage(0, cur);
    bool published_cur = false;   // thread 0's view: cur's flag already set while waiting
    unsigned parity[2] = {0u, 0u};
    for (int it = 0;; ++it) {
        const int cs = it & 1, ns = cs ^ 1;
        const bool has_next = tk_next < total;
        FrogItem nxt = cur;
        if (has_next) {
            nxt = items[tk_next];
            stage(ns, nxt);
        }
        bool published_next = false;
        if (t == 0) {
            s_after = has_next ? atomicAdd(ticket, 1) : total;   // the ticket after next
            if (!mbar_wait(&bars[cs], parity[cs], limit_ns)) {
                atomicCAS(call_err, 0, GNS_ERR_TIMEOUT);
                s_ok = 0;
            } else if (tk != skip_ticket && !published_cur) {
                st_release(&loaded[tk], epoch);         // this chunk's inputs are in shared memory
            }
            if (ld_relaxed(call_err) != 0) s_ok = 0;
            bulk_wait_read_all();                       // the previous chunk's store has read `out`
            if (s_ok && cur.dep_lo <= cur.dep_hi) {
                const unsigned pn = parity[ns];
                auto poll = [&]() {
                    if (!published_next && has_next && tk_next != skip_ticket && mbar_try_wait(&bars[ns], pn)) {
                        st_release(&loaded[tk_next], epoch);
                        published_next = true;
                    }
                };
                bool ok = true;
                for (int32_t q = cur.dep_lo; ok && q <= cur.dep_hi; ++q)
                    ok = wait_flag_polling(&loaded[q], epoch, call_err, limit_ns, poll);
                if (!ok) s_ok = 0;
            }
            fence_proxy_async_global();                 // the bulk store below follows the acquires above
        }
        parity[cs] ^= 1u;
        pending[cs] = false;
        __syncthreads();
        if (!s_ok) break;
        const int64_t tk_after = s_after;
        const StagedChunk g = staged[cs];
        const int cnt = g.na + g.nb;
        uint64_t k[ITEMS];
        uint32_t v[ITEMS];
        const int m = merge_staged<C, ITEMS>(sm.in[cs], g, k, v, has_vals);
        if (m > 0) write_out<C, ITEMS>(sm.out, k, v, m, has_vals, mode, decode_out);
        fence_proxy_async_shared();
        __syncthreads();
        if (cnt > 0) {
            const int64_t o = cur.oslot;
            const bool contiguous = (o + cnt <= sl.n) || (o >= sl.n);
            uint64_t* Dk = sl.kp(o);
            uint32_t* Dv = has_vals ? sl.vp(o) : nullptr;
            if (contiguous && bulk_ok(Dk, Dv, cnt)) {
                if (t == 0) {
                    bulk_store(Dk, sm.out.k, (unsigned)cnt * 8);
                    if (Dv) bulk_store(Dv, sm.out.v, (unsigned)cnt * 4);
                    bulk_commit();
                }
            } else {
                for (int e = t; e < cnt; e += THREADS) {
                    *sl.kp(o + e) = sm.out.k[e];
                    if (Dv) *sl.vp(o + e) = sm.out.v[e];
                }
            }
        }
        if (!has_next) break;
        tk = tk_next;
        tk_next = tk_after;
        cur = nxt;
        published_cur = published_next;
    }
    if (t == 0) {
        bulk_wait_all();
        for (int q = 0; q < 2; ++q)
            if (pending[q]) mbar_wait(&bars[q], parity[q], limit_ns);
    }
}

}  // namespace gns
