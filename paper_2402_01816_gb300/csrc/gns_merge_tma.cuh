// gns_merge_tma.cuh -- building blocks of the merge levels on sm_100+: the
// PTX wrappers for mbarriers and bulk (TMA) copies, the chunk geometry of a
// Nocopy level, the shared-memory stage layout, and the in-place level's work
// items.  The pipelines themselves are in gns_merge_ws.cuh.
//
// Alignment: bulk copies move 16-byte aligned blocks between 16-byte aligned
// addresses; the stages keep a few spare words so that a slice copied from
// the 16-byte boundary at or below its first element still fits.
#pragma once

#include "gns_kernels.cuh"

namespace gns {


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
    uint64_t k[C + 10];   // + spare words: copies rounded out to 16 bytes, and heads read past a run
    uint32_t v[C + 16];
};
template <int C>
struct OutBuf {
    uint64_t k[C + 2];   // room for outputs shifted to the destination's 16-byte phase
    uint32_t v[C + 4];
};
// Where the two input slices of a staged chunk sit in shared memory.
struct StagedChunk {
    int na, nb;
    int ka, kb;   // shared index of the first key of each slice
    int va, vb;   // shared index of the first payload word of each slice
};

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
    int64_t ra, rb;        // lowest slot of the first / second slice (left / right run unless SYM)
    int64_t oslot;         // slot of the first output
    int32_t na, nb;        // slice lengths (0, 0: nothing to do)
    int32_t dep_lo, dep_hi;   // items whose loads must precede the store (dep_hi < dep_lo: none)
    int32_t flags;         // SYM levels: FI_REV_A / FI_REV_B (slice read from its far end), FI_DESC
    int32_t id;            // the item's "loaded" flag: node-major, node k's items at base(k) + local
};
enum { FI_REV_A = 1, FI_REV_B = 2, FI_DESC = 4 };

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

// frog_dep_range for nodes of either orientation (SYM levels).  The outer
// child's run lies under the output and is never read reversed; its consumed
// index i sits at output index i + off (off = 0 for a data-left node, the
// inner child's size for a data-right one) and every element moves towards
// the node's outer end, so only later chunks (data-left) or earlier chunks
// (data-right) can read what chunk c overwrites.  The outer run is the first
// run F (whose counts the splits hold) or the second, by orientation.
__device__ __forceinline__ int2 frog_dep_range_sym(int64_t c, const FrogNode& x, int64_t nF, int64_t n_outer,
                                                   bool outer_is_f, const int64_t* sp, int C)
{
    int2 r = make_int2(0, -1);
    const int64_t w0 = c * C, w1 = imin64(w0 + C, x.n);
    if (w0 >= x.n) return r;
    const int64_t last = (x.n - 1) / C;
    auto f_end = [&](int64_t q) { return q == last ? nF : sp[q + 1]; };
    auto o_beg = [&](int64_t q) { return outer_is_f ? sp[q] : q * C - sp[q]; };
    auto o_end = [&](int64_t q) { return outer_is_f ? f_end(q) : imin64((q + 1) * C, x.n) - f_end(q); };
    const int64_t off = x.side == 0 ? 0 : x.n - n_outer;
    const int64_t lo_o = imax64(w0 - off, 0), hi_o = imin64(w1 - off, n_outer);
    if (lo_o >= hi_o) return r;
    if (x.side == 0) {
        if (c >= last) return r;
        int64_t lo = c + 1, hi = last;                  // first q > c with o_end(q) > lo_o
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (o_end(mid) > lo_o) hi = mid;
            else lo = mid + 1;
        }
        if (o_beg(lo) >= hi_o) return r;
        int64_t lo2 = lo, hi2 = last;                   // last q with o_beg(q) < hi_o
        while (lo2 < hi2) {
            const int64_t mid = (lo2 + hi2 + 1) >> 1;
            if (o_beg(mid) < hi_o) lo2 = mid;
            else hi2 = mid - 1;
        }
        r = make_int2((int)lo, (int)lo2);
    } else {
        if (c <= 0 || o_beg(0) >= hi_o) return r;
        int64_t lo = 0, hi = c - 1;                     // last q < c with o_beg(q) < hi_o
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (o_beg(mid) < hi_o) lo = mid;
            else hi = mid - 1;
        }
        if (o_end(lo) <= lo_o) return r;
        int64_t lo2 = 0, hi2 = lo;                      // first q with o_end(q) > lo_o
        while (lo2 < hi2) {
            const int64_t mid = (lo2 + hi2) >> 1;
            if (o_end(mid) > lo_o) hi2 = mid;
            else lo2 = mid + 1;
        }
        r = make_int2((int)lo2, (int)lo);
    }
    return r;
}

// items[tk] for every ticket tk of a level (after the partition, before the
// merge).  An item is chunk c = nchk - 1 - local of a data-left node k or
// chunk c = local of a data-right one; its flag is id = base(k) + local
// (node-major, as frog_locate numbers them), and the dependency ranges are ids.
// Tickets hand the items out interleaved across the nodes: round j takes
// position j of every node that has more than j chunks.  When every node has
// nch chunk slots (the Frogsort1 tree) ticket tk is local = tk / nnodes of
// node k = tk mod nnodes.  A host-planned tree (cstart: nodes of unequal
// chunk counts) lists each depth's nodes largest first, and iseg holds the
// runs of rounds with one node count as triples (first ticket, first round,
// nodes per round): ticket tk of run t is round j = j_t + (tk - ts_t) / c_t of
// node (tk - ts_t) mod c_t.  Within a node the locals
// come in increasing ticket order, so every item a store waits on holds an
// earlier ticket (no cycle of waits), and consecutive items of one node lie
// a round apart: on a level of many small nodes a store no longer waits on a
// ticket taken just before its own.
//
// skip_identity: a chunk whose outputs all come from one run and already sit
// in their output slots (the leading left-run chunks of a data-left node, the
// trailing right-run chunks of a data-right node, when the runs do not
// overlap) becomes an empty item -- no load, no store.  This is the
// symmetric merge's adaptivity to presorted data ("Symmetric merging"
// section: at most half the data moves).  Such a chunk's inputs are its own
// output slots, which no other chunk writes, so no chunk waits on it.  Off on
// the level that decodes the keys, where every element is rewritten.
template <bool SYM>
__global__ void frog_items_kernel(const FrogNode* __restrict__ level, const FrogNode* __restrict__ child,
                                  int64_t nnodes, int64_t nch, const int64_t* __restrict__ cstart, int64_t total,
                                  const int64_t* __restrict__ splits, FrogItem* __restrict__ items, int* call_err,
                                  const int* presorted, int skip_identity, const int32_t* __restrict__ iseg,
                                  int64_t nseg)
{
    const int64_t tk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tk >= total || skip_all(presorted)) return;
    int64_t k, local, base, nchk;
    if (cstart) {
        int64_t lo = 0, hi = nseg - 1;                  // last run t with ts_t <= tk
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (iseg[3 * mid] <= tk) lo = mid;
            else hi = mid - 1;
        }
        const int64_t off = tk - iseg[3 * lo], cnt = iseg[3 * lo + 2];
        local = iseg[3 * lo + 1] + off / cnt;
        k = off % cnt;
        base = cstart[k];
        nchk = cstart[k + 1] - base;
    } else {
        local = tk / nnodes;
        k = tk - local * nnodes;
        base = k * nch;
        nchk = nch;
    }
    const FrogNode x = level[k];
    const int64_t c = x.side == 0 ? nchk - 1 - local : local;
    FrogItem it;
    it.ra = it.rb = it.oslot = 0;
    it.na = it.nb = 0;
    it.dep_lo = 0;
    it.dep_hi = -1;
    it.flags = 0;
    it.id = (int32_t)(base + local);
    const int64_t w0 = c * CHUNK;
    if (w0 < x.n) {
        const int64_t w1 = imin64(w0 + CHUNK, x.n);
        const FrogNode L = child[2 * k], R = child[2 * k + 1];
        // SYM: slice A is the first run F, slice B the second (frog_partition_kernel)
        const bool desc = SYM && x.ori != 0;
        const FrogNode& F = desc ? R : L;
        const FrogNode& S = desc ? L : R;
        const bool rf = SYM && F.ori != x.ori, rs = SYM && S.ori != x.ori;
        const int64_t* sp = splits + base;
        const int64_t a0 = sp[c];
        const int64_t a1 = (w1 == x.n) ? F.n : sp[c + 1];
        const int64_t na = a1 - a0, nb = (w1 - a1) - (w0 - a0);
        if (na < 0 || nb < 0 || na + nb > CHUNK || a0 < 0 || a1 > F.n) {   // splits inconsistent
            atomicCAS(call_err, 0, GNS_ERR_INTERNAL);
        } else {
            it.na = (int32_t)na;
            it.nb = (int32_t)nb;
            it.ra = rf ? frog_data_slot(F) + F.n - a1 : frog_data_slot(F) + a0;
            it.rb = rs ? frog_data_slot(S) + S.n - (w1 - a1) : frog_data_slot(S) + (w0 - a0);
            it.oslot = frog_data_slot(x) + w0;
            it.flags = (rf ? FI_REV_A : 0) | (rs ? FI_REV_B : 0) | (desc ? FI_DESC : 0);
            const bool identity = (nb == 0 && !rf && it.ra == it.oslot) || (na == 0 && !rs && it.rb == it.oslot);
            if (skip_identity && identity) {
                it.na = it.nb = 0;
            } else {
                int2 r;
                if (SYM) {
                    const FrogNode& O = x.side == 0 ? L : R;
                    r = frog_dep_range_sym(c, x, F.n, O.n, (x.side == 0) != desc, sp, CHUNK);
                } else {
                    r = frog_dep_range(c, x, L, R, sp, CHUNK);
                }
                if (r.x <= r.y) {
                    it.dep_lo = (int32_t)(x.side == 0 ? base + nchk - 1 - r.y : base + r.x);
                    it.dep_hi = (int32_t)(x.side == 0 ? base + nchk - 1 - r.x : base + r.y);
                }
            }
        }
    }
    items[tk] = it;
}

}  // namespace gns
