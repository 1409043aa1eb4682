// gns_merge_ws.cuh -- merge levels as warp-specialised TMA pipelines (sm_100+).
//
// A CTA is one producer warp plus CT consumer threads sharing a ring of S
// shared-memory stages.  Lane 0 of the producer warp does everything that
// touches global memory:
//   * takes work items in order (a static stride for the ping-pong levels,
//     tickets for the in-place level) and stages each item's two input slices
//     into the next stage with cp.async.bulk (completion on the stage's "full"
//     mbarrier);
//   * stores each merged chunk from its stage with cp.async.bulk once the
//     consumers have written it (the stage's "done" mbarrier) and -- in the
//     in-place level -- once every item that reads the elements under the
//     chunk's output has published its "inputs loaded" flag;
//   * reuses a stage once its store has read it.
// The consumers merge: wait for a stage (in the in-place level the first
// consumer thread then publishes the item's "inputs loaded" flag), split it by
// merge path (MERGE_ITEMS = 9 outputs per thread), merge serially in registers, and -- after
// a barrier, since the stage is their input -- write the outputs back into the
// same stage,
// placed so that shared and global addresses agree modulo 16 bytes (one bulk
// store for the aligned interior, plain stores for at most 1 key / 3 payload
// words at each end).  The consumers never wait on another CTA, and the
// producer's latency chain (item record, copy issue, flag traffic) runs beside
// the merging.
//
// Termination and errors.  Every wait is bounded.  The consumers leave the
// loop only on decisions that are uniform across them (taken after a named
// barrier from values written before it), so none is left at a barrier.  The
// producer stops on an error, tells the consumers through an abort word, and
// before it exits waits (bounded) for the copies it has in flight.
#pragma once

#include "gns_merge_tma.cuh"

namespace gns {

constexpr int WS_CONSUMERS = MERGE_CONSUMERS;
constexpr int WS_ITEMS = MERGE_ITEMS;
constexpr int WS_CHUNK = CHUNK;                     // outputs per item (the stages hold one)
static_assert(WS_CONSUMERS * WS_ITEMS >= WS_CHUNK, "merge chunk size");

// Resident CTAs per SM the S-stage layouts are sized for (shared memory and
// registers): six 160-thread CTAs with 1024-output stages, three 288-thread
// CTAs with 2048-output stages.
template <int S>
constexpr int ws_ctas_per_sm() { return WS_CONSUMERS == 128 ? (S <= 3 ? 6 : 4) : (S == 2 ? 3 : 2); }
// The in-place level has no out buffer: three of its 3-stage CTAs still fit an
// SM (3 x 74 KB of stages).
template <int S>
constexpr int ws_frog_ctas_per_sm() { return WS_CONSUMERS == 128 ? (S <= 3 ? 6 : 4) : (S <= 3 ? 3 : 2); }

template <int C, int S>
struct WsSmem {
    InStage<C> in[S];
};

// One item as the producer stages it.
struct WsLoad {
    const uint64_t* ak; const uint32_t* av; int na;
    const uint64_t* bk; const uint32_t* bv; int nb;
    const uint64_t* ak_end; const uint32_t* av_end;   // ends of the arrays holding the slices: a copy
    const uint64_t* bk_end; const uint32_t* bv_end;   // rounded out to 16 bytes must stay below them
    bool plain_a, plain_b;        // slice straddles the caller-array / buffer boundary (slot addressing)
    int64_t slot_a, slot_b;
    uint64_t* dk; uint32_t* dv;   // contiguous destination, or dk == nullptr: store by slots from oslot
    int64_t oslot;
    int decode;
    int64_t tk;                   // item index (in-place level: its "loaded" flag)
    int32_t dep_lo, dep_hi;       // items whose loads must precede the store
    int flags;                    // FrogItem::flags (symmetric in-place levels)
};

// What the consumers need of a staged item.
struct WsInfo {
    StagedChunk g;
    int shk, shv;                 // outputs start at shared index shk (keys) / shv (payload)
    int decode;
    int end;                      // no more items
    int64_t tk;                   // in-place level: the item's "loaded" flag
    int flags;                    // FrogItem::flags (symmetric in-place levels)
};

// What the producer keeps of a staged item until its store.
struct WsOut {
    uint64_t* dk; uint32_t* dv;
    int64_t oslot;
    int cnt, shk, shv;
};

// Non-blocking test of an mbarrier phase (try_wait may suspend the thread for a
// while; the producer's event loop must not).
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void named_bar_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// Wait until at most n of this thread's bulk store groups still read shared memory.
__device__ __forceinline__ void bulk_wait_read_n(int n)
{
    switch (n) {
    case 0: asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.bulk.wait_group.read 2;" ::: "memory"); break;
    default: asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory"); break;
    }
}

// One input slice staged by a single thread: one bulk copy from the 16-byte
// boundary at or below its first element to the boundary at or above its end
// when that stays inside the array (returns the byte count), else a copy to
// the boundary below the end plus plain loads of the at most one key / three
// payload words after it; or, for a slice addressed by slots, plain loads.
__device__ __forceinline__ unsigned stage_slice_1t(uint64_t* sk, uint32_t* svv, int s0k, int s0v,
                                                   const uint64_t* P, const uint32_t* Pv, int m, uint64_t* bar,
                                                   int& koff, int& voff, const Slots* plain_sl, int64_t plain_slot,
                                                   bool has_vals, const uint64_t* Pend, const uint32_t* Pvend)
{
    unsigned bytes = 0;
    if (plain_sl) {
        koff = s0k;
        voff = s0v;
        for (int e = 0; e < m; ++e) {
            sk[s0k + e] = *plain_sl->kp(plain_slot + e);
            if (has_vals) svv[s0v + e] = *plain_sl->vp(plain_slot + e);
        }
        return 0;
    }
    if (m == 0) {
        koff = s0k;
        voff = s0v;
        return 0;
    }
    const uintptr_t pk = (uintptr_t)P, pk_lo = pk & ~(uintptr_t)15, pk_end = pk + (uintptr_t)m * 8;
    const uintptr_t pk_up = (pk_end + 15) & ~(uintptr_t)15;
    const uintptr_t pk_hi = pk_up <= (uintptr_t)Pend ? pk_up : (pk_end & ~(uintptr_t)15);
    koff = s0k + (int)((pk - pk_lo) >> 3);
    if (pk_hi > pk_lo) {
        bulk_load(sk + s0k, (const void*)pk_lo, (unsigned)(pk_hi - pk_lo), bar);
        bytes += (unsigned)(pk_hi - pk_lo);
    }
    if (pk_hi < pk_end) {                            // the rounded copy would leave the array
        const int ktail = pk_hi > pk ? (int)((pk_hi - pk) >> 3) : 0;
        for (int e = ktail; e < m; ++e) sk[koff + e] = P[e];
    }
    voff = s0v;
    if (has_vals) {
        const uintptr_t pv = (uintptr_t)Pv, pv_lo = pv & ~(uintptr_t)15, pv_end = pv + (uintptr_t)m * 4;
        const uintptr_t pv_up = (pv_end + 15) & ~(uintptr_t)15;
        const uintptr_t pv_hi = pv_up <= (uintptr_t)Pvend ? pv_up : (pv_end & ~(uintptr_t)15);
        voff = s0v + (int)((pv - pv_lo) >> 2);
        if (pv_hi > pv_lo) {
            bulk_load(svv + s0v, (const void*)pv_lo, (unsigned)(pv_hi - pv_lo), bar);
            bytes += (unsigned)(pv_hi - pv_lo);
        }
        if (pv_hi < pv_end) {
            const int vtail = pv_hi > pv ? (int)((pv_hi - pv) >> 2) : 0;
            for (int e = vtail; e < m; ++e) svv[voff + e] = Pv[e];
        }
    }
    return bytes;
}

// Merge of a staged chunk by consumer thread `ct`: its outputs [ITEMS ct, ITEMS ct + ITEMS).
template <int C, int ITEMS>
__device__ __forceinline__ int merge_staged_ct(const InStage<C>& st, const StagedChunk& g, uint64_t (&k)[ITEMS],
                                               uint32_t (&v)[ITEMS], bool has_vals, int ct)
{
    const int na = g.na, nb = g.nb, cnt = na + nb;
    const int diag = ct * ITEMS;
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
    // "take A" tests both bounds itself, so a head is reloaded without a bounds
    // test: past run A it reads at most ITEMS words past it (slice B or the
    // stage's spare words: run A starts at word 0 or 1 and is shorter than C),
    // past run B at most its next word.  Such a value is never used.
#pragma unroll
    for (int x = 0; x < ITEMS; ++x) {
        const bool takeA = (j >= nb) || (i < na && ka <= kb);
        k[x] = takeA ? ka : kb;
        if (has_vals) v[x] = takeA ? st.v[g.va + (i < na ? i : na - 1)] : st.v[g.vb + (j < nb ? j : nb - 1)];
        if (takeA) {
            ++i;
            ka = st.k[g.ka + i];
        } else {
            ++j;
            kb = st.k[g.kb + j];
        }
    }
    return cnt - diag < ITEMS ? cnt - diag : ITEMS;
}

// merge_staged_ct for the symmetric in-place levels (nodes of either
// orientation, frog_partition_kernel): slice A is the first run, and a slice
// flagged FI_REV_* is consumed from its highest slot down; keys are compared
// after XOR with the mask (all ones for a mirrored node, whose slot order puts
// larger keys first), the stored keys are unchanged.  As in merge_staged_ct a
// head is reloaded without a bounds test: one word past the end of a run, which
// for a reversed slice is the word below it -- the symmetric levels stage
// their slices from word SYM_STAGE_K0 on, so that word is inside the stage.
// (Items without flags take merge_staged_ct itself.)
constexpr int SYM_STAGE_K0 = 2, SYM_STAGE_V0 = 4;   // first staged key / payload word (16-byte aligned)
template <int C, int ITEMS>
__device__ __forceinline__ int merge_staged_sym(const InStage<C>& st, const StagedChunk& g, int flags,
                                                uint64_t (&k)[ITEMS], uint32_t (&v)[ITEMS], bool has_vals, int ct)
{
    const int na = g.na, nb = g.nb, cnt = na + nb;
    const int diag = ct * ITEMS;
    if (diag >= cnt) return 0;
    const uint64_t mask = (flags & FI_DESC) ? ~0ull : 0ull;
    const int sa = (flags & FI_REV_A) ? -1 : 1, sb = (flags & FI_REV_B) ? -1 : 1;
    const int pa = (flags & FI_REV_A) ? g.ka + na - 1 : g.ka, pb = (flags & FI_REV_B) ? g.kb + nb - 1 : g.kb;
    const int qa = (flags & FI_REV_A) ? g.va + na - 1 : g.va, qb = (flags & FI_REV_B) ? g.vb + nb - 1 : g.vb;
    int lo = diag - nb > 0 ? diag - nb : 0, hi = diag < na ? diag : na;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((st.k[pa + sa * mid] ^ mask) <= (st.k[pb + sb * (diag - 1 - mid)] ^ mask)) lo = mid + 1;
        else hi = mid;
    }
    int i = lo, j = diag - lo;
    int xa = pa + sa * i, xb = pb + sb * j;          // shared index of each run's head
    int ya = qa + sa * i, yb = qb + sb * j;
    uint64_t ka = i < na ? st.k[xa] ^ mask : ~0ull;
    uint64_t kb = j < nb ? st.k[xb] ^ mask : ~0ull;
#pragma unroll
    for (int x = 0; x < ITEMS; ++x) {
        const bool takeA = (j >= nb) || (i < na && ka <= kb);
        k[x] = (takeA ? ka : kb) ^ mask;
        if (has_vals) v[x] = st.v[takeA ? ya : yb];
        if (takeA) {
            ++i;
            xa += sa;
            ya += sa;
            ka = st.k[xa] ^ mask;
        } else {
            ++j;
            xb += sb;
            yb += sb;
            kb = st.k[xb] ^ mask;
        }
    }
    return cnt - diag < ITEMS ? cnt - diag : ITEMS;
}

// copy_staged_striped for the symmetric in-place levels: the one non-empty
// slice, consumed from its far end when flagged.
template <int C, int ITEMS, int CT>
__device__ __forceinline__ void copy_staged_sym(const InStage<C>& st, const StagedChunk& g, int flags,
                                                uint64_t (&k)[ITEMS], uint32_t (&v)[ITEMS], bool has_vals, int ct)
{
    const bool from_a = g.nb == 0;
    const int cnt = g.na + g.nb;
    const bool rev = (flags & (from_a ? FI_REV_A : FI_REV_B)) != 0;
    const int bk = from_a ? g.ka : g.kb, bv = from_a ? g.va : g.vb;
#pragma unroll
    for (int x = 0; x < ITEMS; ++x) {
        const int e = ct + x * CT;
        if (e < cnt) {
            const int q = rev ? cnt - 1 - e : e;
            k[x] = st.k[bk + q];
            if (has_vals) v[x] = st.v[bv + q];
        }
    }
}

// A chunk whose outputs all come from one run (one slice empty: presorted
// stretches) is a copy: consumer thread ct takes outputs ct, ct + CT, ...
// (striped, so a warp's accesses are consecutive words: no bank conflicts).
template <int C, int ITEMS, int CT>
__device__ __forceinline__ void copy_staged_striped(const InStage<C>& st, const StagedChunk& g, uint64_t (&k)[ITEMS],
                                                    uint32_t (&v)[ITEMS], bool has_vals, int ct)
{
    const bool from_a = g.nb == 0;
    const int bk = from_a ? g.ka : g.kb, bv = from_a ? g.va : g.vb, cnt = g.na + g.nb;
#pragma unroll
    for (int x = 0; x < ITEMS; ++x) {
        const int e = ct + x * CT;
        if (e < cnt) {
            k[x] = st.k[bk + e];
            if (has_vals) v[x] = st.v[bv + e];
        }
    }
}

template <int ITEMS, int CT>
__device__ __forceinline__ void write_striped_shifted(uint64_t* ok, uint32_t* ov, int shk, int shv,
                                                     const uint64_t (&k)[ITEMS], const uint32_t (&v)[ITEMS], int cnt,
                                                     bool has_vals, int mode, int decode_out, int ct)
{
#pragma unroll
    for (int x = 0; x < ITEMS; ++x) {
        const int e = ct + x * CT;
        if (e < cnt) {
            ok[shk + e] = decode_out ? decode_key(k[x], mode) : k[x];
            if (has_vals) ov[shv + e] = v[x];
        }
    }
}

// a[y] <- a[(y + r) mod N] (N a power of two, 0 <= r < N): log2(N) stages of
// conditional fixed rotations, so no register is indexed at run time.
template <int N, typename T>
__device__ __forceinline__ void rotate_left(T (&a)[N], int r)
{
#pragma unroll
    for (int sft = 1; sft < N; sft <<= 1) {
        const bool on = (r & sft) != 0;
        T tmp[N];
#pragma unroll
        for (int y = 0; y < N; ++y) tmp[y] = a[(y + sft) & (N - 1)];
#pragma unroll
        for (int y = 0; y < N; ++y) a[y] = on ? tmp[y] : a[y];
    }
}

// Thread ct's m outputs to keys ok[shk + ITEMS ct ...] and payload
// ov[shv + ITEMS ct ...].  With an odd ITEMS the threads' blocks start an odd
// number of payload words (and twice that many key words) apart, so a store
// step of all threads hits distinct banks as it is.  With ITEMS = 8 a full set
// of outputs is written one element per store in a rotated order: at step y
// thread ct writes its element (y + r) mod 8, r = ct / 2 for keys and ct / 4
// for the payload, so that within a half-warp (8-byte keys) the 16 threads'
// slots ((8 ct + element) mod 16) are all different, and so are the 32
// threads' payload banks ((8 ct + element) mod 32), whatever the shift.
template <int ITEMS>
__device__ __forceinline__ void write_out_shifted(uint64_t* ok, uint32_t* ov, int shk, int shv,
                                                  uint64_t (&kk)[ITEMS], uint32_t (&v)[ITEMS], int m,
                                                  bool has_vals, int mode, int decode_out, int ct)
{
    const int diag = ct * ITEMS;
    if (decode_out) {
#pragma unroll
        for (int x = 0; x < ITEMS; ++x) kk[x] = decode_key(kk[x], mode);
    }
    if (m == ITEMS) {
        if constexpr ((ITEMS & 1) != 0) {
            // an odd count: thread blocks start 2*ITEMS words apart (keys) and
            // ITEMS words apart (payload), distinct banks with no rotation
#pragma unroll
            for (int y = 0; y < ITEMS; ++y) {
                ok[shk + diag + y] = kk[y];
                if (has_vals) ov[shv + diag + y] = v[y];
            }
        } else {
            static_assert(ITEMS == 8, "rotated write-out assumes 8 outputs per thread");
            uint64_t* dk = ok + shk + diag;
            const int rk = (ct >> 1) & 7;
            rotate_left<ITEMS>(kk, rk);
#pragma unroll
            for (int y = 0; y < ITEMS; ++y) dk[(y + rk) & 7] = kk[y];
            if (has_vals) {
                uint32_t* dv = ov + shv + diag;
                const int rv = (ct >> 2) & 7;
                rotate_left<ITEMS>(v, rv);
#pragma unroll
                for (int y = 0; y < ITEMS; ++y) dv[(y + rv) & 7] = v[y];
            }
        }
    } else {
#pragma unroll
        for (int x = 0; x < ITEMS; ++x) {
            if (x < m) {
                ok[shk + diag + x] = kk[x];
                if (has_vals) ov[shv + diag + x] = v[x];
            }
        }
    }
}

// Bounded wait for an mbarrier phase that also gives up when *abort is set.
__device__ __forceinline__ bool mbar_wait_abortable(uint64_t* bar, unsigned parity, uint64_t limit_ns,
                                                    const volatile int* abort)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// Stores a merged chunk from its stage (producer thread): one bulk store per
// array for the 16-byte-aligned interior, plain stores for the ends; a chunk
// whose destination changes arrays (dk == nullptr) goes element by element
// through the slots.  Commits one bulk group (possibly empty).
__device__ __forceinline__ void ws_store(const uint64_t* sk, const uint32_t* sv, const WsOut& o, const Slots& sl,
                                         bool has_vals)
{
    const int cnt = o.cnt;
    if (cnt > 0 && o.dk == nullptr) {
        for (int e = 0; e < cnt; ++e) {
            *sl.kp(o.oslot + e) = sk[o.shk + e];
            if (has_vals) *sl.vp(o.oslot + e) = sv[o.shv + e];
        }
    } else if (cnt > 0) {
        // keys: element e at sk[shk + e]; global dk + e is 16-byte aligned for e = shk mod 2
        const int klo = o.shk < cnt ? o.shk : cnt;
        const int khi = klo + ((cnt - klo) & ~1);
        if (khi > klo) bulk_store(o.dk + klo, &sk[o.shk + klo], (unsigned)(khi - klo) * 8);
        for (int e = 0; e < klo; ++e) o.dk[e] = sk[o.shk + e];
        for (int e = khi; e < cnt; ++e) o.dk[e] = sk[o.shk + e];
        if (has_vals) {
            const int l0 = (4 - o.shv) & 3;
            const int vlo = l0 < cnt ? l0 : cnt;
            const int vhi = vlo + ((cnt - vlo) & ~3);
            if (vhi > vlo) bulk_store(o.dv + vlo, &sv[o.shv + vlo], (unsigned)(vhi - vlo) * 4);
            for (int e = 0; e < vlo; ++e) o.dv[e] = sv[o.shv + e];
            for (int e = vhi; e < cnt; ++e) o.dv[e] = sv[o.shv + e];
        }
    }
    bulk_commit();
}

// Shifts that make shared index (e + shk) and global dk + e agree modulo 16
// bytes (and likewise for the payload).
__device__ __forceinline__ void ws_shifts(const uint64_t* dk, const uint32_t* dv, int& shk, int& shv)
{
    shk = dk ? (int)(((uintptr_t)dk >> 3) & 1) : 0;
    shv = (dk && dv) ? (int)(((uintptr_t)dv >> 2) & 3) : 0;
}

// The pipeline.  Src::next(WsLoad&) hands the producer its next item (false:
// none left).  FLAGS: publish/await "inputs loaded" flags (in-place level).
template <int CT, int ITEMS, int S, bool FLAGS, bool SYM, typename Src>
__device__ __forceinline__ void ws_merge(Src& src, const Slots& sl, bool has_vals, int mode, int* call_err,
                                         uint64_t limit_ns, int* loaded, int epoch, int64_t skip_ticket,
                                         uint32_t jitter_ns)
{
    constexpr int C = WS_CHUNK;
    static_assert(S >= 2 && S <= 4 && CT * ITEMS >= C, "stages");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    WsSmem<C, S>& sm = *reinterpret_cast<WsSmem<C, S>*>(smem_raw);
    __shared__ __align__(8) uint64_t full[S];
    __shared__ __align__(8) uint64_t done[S];
    __shared__ WsInfo info[S];
    __shared__ volatile int s_pabort;
    __shared__ volatile int s_cfail;
    const int t = threadIdx.x;
    if (t == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&done[q], CT / 32);           // one arrival per consumer warp
        }
        s_pabort = 0;
        s_cfail = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (t < 32) {
        // ------------------------------------------------------------ producer
        if (t != 0) return;
        WsOut out[S];
        int32_t sdn[S], sdh[S];
        int64_t n_staged = 0;    // items staged (item i uses stage i % S)
        int64_t n_stored = 0;    // items whose store has been issued (in item order)
        bool no_more = false;
        bool failed = false;
        uint64_t t_last = global_ns();
        for (;;) {
            bool progress = false;
            // store merged chunks, in item order
            while (n_stored < n_staged) {
                const int q = (int)(n_stored % S);
                if (!mbar_test(&done[q], (unsigned)(n_stored / S) & 1u)) break;
                if (FLAGS) {
                    bool ok = true;
                    while (sdn[q] <= sdh[q]) {
                        if (ld_acquire(&loaded[sdn[q]]) != epoch) {
                            ok = false;
                            break;
                        }
                        ++sdn[q];
                    }
                    if (!ok) break;
                    fence_proxy_async_global();      // the store below follows the acquires above
                }
                ws_store(sm.in[q].k, sm.in[q].v, out[q], sl, has_vals);
                ++n_stored;
                progress = true;
            }
            // stage the next item once its stage's previous store has read it
            if (!no_more) {
                const int64_t i = n_staged;
                const int q = (int)(i % S);
                bool free_ = i < S;
                if (!free_ && n_stored > i - S) {
                    bulk_wait_read_n((int)(n_stored - 1 - (i - S)));
                    free_ = true;
                }
                if (free_) {
                    WsLoad L;
                    if (ld_relaxed(call_err) != 0 || !src.next(L)) {
                        info[q].end = 1;
                        mbar_arrive(&full[q]);
                        no_more = true;
                    } else {
                        int na = L.na, nb = L.nb;
                        if (na < 0 || nb < 0 || na + nb > C) {   // inconsistent item: stage nothing
                            atomicCAS(call_err, 0, GNS_ERR_INTERNAL);
                            na = nb = 0;
                        }
                        debug_jitter(jitter_ns, L.tk, epoch);  // test hook: the held ticket loads late
                        fence_proxy_async_shared();            // earlier accesses of this stage come first
                        WsInfo inf;
                        inf.g.na = na;
                        inf.g.nb = nb;
                        InStage<C>& st = sm.in[q];
                        // symmetric levels: two spare key words below slice A (merge_staged_sym)
                        unsigned bytes = stage_slice_1t(st.k, st.v, SYM ? SYM_STAGE_K0 : 0, SYM ? SYM_STAGE_V0 : 0,
                                                        L.ak, L.av, na, &full[q], inf.g.ka, inf.g.va,
                                                        L.plain_a ? &sl : nullptr, L.slot_a, has_vals, L.ak_end,
                                                        L.av_end);
                        const int s0k = (inf.g.ka + na + 1) & ~1;     // 16-byte boundary after slice A
                        const int s0v = (inf.g.va + na + 3) & ~3;
                        bytes += stage_slice_1t(st.k, st.v, s0k, s0v, L.bk, L.bv, nb, &full[q], inf.g.kb, inf.g.vb,
                                                L.plain_b ? &sl : nullptr, L.slot_b, has_vals, L.bk_end, L.bv_end);
                        WsOut o;
                        o.dk = L.dk;
                        o.dv = L.dv;
                        o.oslot = L.oslot;
                        o.cnt = na + nb;
                        ws_shifts(L.dk, L.dv, o.shk, o.shv);
                        out[q] = o;
                        inf.shk = o.shk;
                        inf.shv = o.shv;
                        inf.decode = L.decode;
                        inf.end = 0;
                        inf.tk = L.tk;
                        inf.flags = L.flags;
                        info[q] = inf;
                        sdn[q] = L.dep_lo;
                        sdh[q] = L.dep_hi;
                        ++n_staged;
                        mbar_arrive_expect_tx(&full[q], bytes);   // the arrival: the phase ends when the bytes land
                    }
                    progress = true;
                }
            }
            if (no_more && n_stored == n_staged) break;
            if (progress) {
                t_last = global_ns();
            } else {
                if (ld_relaxed(call_err) != 0 || s_cfail) { failed = true; break; }
                if (global_ns() - t_last > limit_ns) {
                    atomicCAS(call_err, 0, GNS_ERR_TIMEOUT);
                    failed = true;
                    break;
                }
                __nanosleep(64);                     // keep the polling off the shared-memory pipe
            }
        }
        if (failed) s_pabort = 1;
        // copies in flight must end before the CTA does
        bulk_wait_all();
        for (int64_t i = n_stored; i < n_staged; ++i) mbar_wait(&full[i % S], (unsigned)(i / S) & 1u, limit_ns);
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int ct = t - 32;
    for (int64_t i = 0;; ++i) {
        const int s = (int)(i % S);
        const unsigned ph = (unsigned)(i / S) & 1u;
        const bool ok = mbar_wait_abortable(&full[s], ph, limit_ns, &s_pabort);
        if (!ok) {
            if (!s_pabort) atomicCAS(call_err, 0, GNS_ERR_TIMEOUT);
            s_cfail = 1;
        }
        const WsInfo inf = info[s];
        // publish the item's "inputs loaded" flag as soon as its stage has landed
        // (a consumer thread has no global stores outstanding, so the release is cheap)
        if (FLAGS && ct == 0 && ok && !inf.end && inf.tk != skip_ticket) st_release(&loaded[inf.tk], epoch);
        uint64_t k[ITEMS];
        uint32_t v[ITEMS];
        int m = 0;
        const bool one = inf.g.na == 0 || inf.g.nb == 0;   // uniform: from the stage's record
        if (ok && !inf.end) {
            if (SYM && inf.flags != 0) {       // uniform: from the stage's record
                if (one) copy_staged_sym<C, ITEMS, CT>(sm.in[s], inf.g, inf.flags, k, v, has_vals, ct);
                else m = merge_staged_sym<C, ITEMS>(sm.in[s], inf.g, inf.flags, k, v, has_vals, ct);
            } else {
                if (one) copy_staged_striped<C, ITEMS, CT>(sm.in[s], inf.g, k, v, has_vals, ct);
                else m = merge_staged_ct<C, ITEMS>(sm.in[s], inf.g, k, v, has_vals, ct);
            }
        }
        named_bar_sync(1, CT);                       // every consumer is done reading the stage
        if (s_cfail || inf.end) break;               // uniform: written before the barrier
        if (one)
            write_striped_shifted<ITEMS, CT>(sm.in[s].k, sm.in[s].v, inf.shk, inf.shv, k, v, inf.g.na + inf.g.nb,
                                             has_vals, mode, inf.decode, ct);
        else if (m > 0)
            write_out_shifted<ITEMS>(sm.in[s].k, sm.in[s].v, inf.shk, inf.shv, k, v, m, has_vals, mode, inf.decode,
                                     ct);
        fence_proxy_async_shared();
        __syncwarp();
        if ((ct & 31) == 0) mbar_arrive(&done[s]);
    }
}

// The pipeline for levels whose items do not depend on one another (ping-pong
// and segmented levels): S input stages plus one out buffer; the producer only
// stages, and consumer thread 0 stores each chunk from the out buffer.  A stage
// goes back to the producer as soon as the consumers have merged it, so the
// next load overlaps the write-out and the store.
template <int C, int S>
struct WsSmemOut {
    InStage<C> in[S];
    OutBuf<C> out;
};

template <int CT, int ITEMS, int S, typename Src>
__device__ __forceinline__ void ws_merge_out(Src& src, bool has_vals, int mode, int* call_err, uint64_t limit_ns)
{
    constexpr int C = WS_CHUNK;
    static_assert(CT * ITEMS >= C, "consumers cover a chunk");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    WsSmemOut<C, S>& sm = *reinterpret_cast<WsSmemOut<C, S>*>(smem_raw);
    __shared__ __align__(8) uint64_t full[S];
    __shared__ __align__(8) uint64_t freeb[S];
    __shared__ WsInfo info[S];
    __shared__ WsOut dst[S];
    __shared__ volatile int s_pabort;
    __shared__ volatile int s_cfail;
    const int t = threadIdx.x;
    if (t == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&freeb[q], 1);
        }
        s_pabort = 0;
        s_cfail = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (t < 32) {
        // ------------------------------------------------------------ producer
        if (t != 0) return;
        int64_t i = 0;
        bool aborted = false;
        for (;; ++i) {
            const int q = (int)(i % S);
            if (i >= S && !mbar_wait_abortable(&freeb[q], (unsigned)((i / S) - 1) & 1u, limit_ns, &s_cfail)) {
                if (!s_cfail) atomicCAS(call_err, 0, GNS_ERR_TIMEOUT);
                s_pabort = 1;
                aborted = true;
                break;
            }
            WsLoad L;
            if (ld_relaxed(call_err) != 0 || !src.next(L)) {
                info[q].end = 1;
                mbar_arrive(&full[q]);
                break;
            }
            int na = L.na, nb = L.nb;
            if (na < 0 || nb < 0 || na + nb > C) {   // inconsistent item: stage nothing
                atomicCAS(call_err, 0, GNS_ERR_INTERNAL);
                na = nb = 0;
            }
            fence_proxy_async_shared();               // the consumers' reads of this stage come first
            WsInfo inf;
            inf.g.na = na;
            inf.g.nb = nb;
            InStage<C>& st = sm.in[q];
            unsigned bytes = stage_slice_1t(st.k, st.v, 0, 0, L.ak, L.av, na, &full[q], inf.g.ka, inf.g.va, nullptr,
                                            0, has_vals, L.ak_end, L.av_end);
            const int s0k = (inf.g.ka + na + 1) & ~1;
            const int s0v = (inf.g.va + na + 3) & ~3;
            bytes += stage_slice_1t(st.k, st.v, s0k, s0v, L.bk, L.bv, nb, &full[q], inf.g.kb, inf.g.vb, nullptr, 0,
                                    has_vals, L.bk_end, L.bv_end);
            WsOut o;
            o.dk = L.dk;
            o.dv = L.dv;
            o.oslot = 0;
            o.cnt = na + nb;
            ws_shifts(L.dk, L.dv, o.shk, o.shv);
            inf.shk = o.shk;
            inf.shv = o.shv;
            inf.decode = L.decode;
            inf.end = 0;
            info[q] = inf;
            dst[q] = o;
            mbar_arrive_expect_tx(&full[q], bytes);
        }
        // copies still landing in shared memory must end before the CTA does.
        // Items before i - S + 1 were merged (their stages came back); item
        // i - S too unless the loop stopped waiting for its stage.  (Parity
        // waits cannot tell phases two apart, so a stage that took the end
        // marker is not waited on again.)
        const int64_t first = aborted ? (i >= S ? i - S : 0) : (i >= S ? i - S + 1 : 0);
        for (int64_t j = first; j < i; ++j) mbar_wait(&full[j % S], (unsigned)(j / S) & 1u, limit_ns);
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int ct = t - 32;
    const Slots none{};
    for (int64_t i = 0;; ++i) {
        const int s = (int)(i % S);
        const unsigned ph = (unsigned)(i / S) & 1u;
        const bool ok = mbar_wait_abortable(&full[s], ph, limit_ns, &s_pabort);
        if (!ok) {
            if (!s_pabort) atomicCAS(call_err, 0, GNS_ERR_TIMEOUT);
            s_cfail = 1;
        }
        const WsInfo inf = info[s];
        WsOut o;
        if (ct == 0) o = dst[s];                      // read before the stage goes back to the producer
        uint64_t k[ITEMS];
        uint32_t v[ITEMS];
        int m = 0;
        const bool one = inf.g.na == 0 || inf.g.nb == 0;   // uniform: from the stage's record
        if (ok && !inf.end) {
            if (one) copy_staged_striped<C, ITEMS, CT>(sm.in[s], inf.g, k, v, has_vals, ct);
            else m = merge_staged_ct<C, ITEMS>(sm.in[s], inf.g, k, v, has_vals, ct);
        }
        if (ct == 0) bulk_wait_read_all();           // the previous store has read `out`
        named_bar_sync(1, CT);
        if (s_cfail || inf.end) break;               // uniform: written before the barrier
        if (ct == 0) mbar_arrive(&freeb[s]);          // every consumer is done with the stage
        if (one)
            write_striped_shifted<ITEMS, CT>(sm.out.k, sm.out.v, inf.shk, inf.shv, k, v, inf.g.na + inf.g.nb,
                                             has_vals, mode, inf.decode, ct);
        else if (m > 0)
            write_out_shifted<ITEMS>(sm.out.k, sm.out.v, inf.shk, inf.shv, k, v, m, has_vals, mode, inf.decode, ct);
        fence_proxy_async_shared();
        named_bar_sync(1, CT);
        if (ct == 0) ws_store(sm.out.k, sm.out.v, o, none, has_vals);
    }
    if (ct == 0) bulk_wait_all();
}

// ------------------------------------------------------------ item sources
// Nocopy level of the 100% tier: chunk b of runs of width w, b = blockIdx.x,
// blockIdx.x + gridDim.x, ...
template <int C>
struct PlainLevelSrc {
    const uint64_t* sk; const uint32_t* sv; uint64_t* dk; uint32_t* dv;
    int64_t n, w, nblocks;
    const int64_t* splits;
    int decode;
    int64_t b;
    __device__ __forceinline__ bool next(WsLoad& L)
    {
        if (b >= nblocks) return false;
        const ChunkGeo g = merge_chunk_geo<C>(b, n, w, splits);
        L.ak = sk + g.a_src; L.av = sv ? sv + g.a_src : nullptr; L.na = g.na;
        L.bk = sk + g.b_src; L.bv = sv ? sv + g.b_src : nullptr; L.nb = g.nb;
        L.ak_end = L.bk_end = sk + n;
        L.av_end = L.bv_end = sv ? sv + n : nullptr;
        L.plain_a = L.plain_b = false;
        L.slot_a = L.slot_b = 0;
        L.dk = dk + g.out0; L.dv = dv ? dv + g.out0 : nullptr;
        L.oslot = 0;
        L.decode = decode;
        L.tk = 0;
        L.dep_lo = 0;
        L.dep_hi = -1;
        L.flags = 0;
        b += gridDim.x;
        return true;
    }
};

// In-place level of the <= 50% tier: items by ticket (see frog_items_kernel
// for the order).  A ticket is taken only when a stage is free and is staged
// at once: a ticket held but not yet loaded would hold up every later item
// whose store waits on it (measured: several times slower on nearly sorted
// input).  Waits only go to earlier tickets, and every taken ticket's inputs
// are loaded and published without waiting on anything, so no cycle of waits
// can form.
struct FrogLevelSrc {
    Slots sl;
    const FrogItem* items;
    int64_t total;
    int* ticket;
    int decode;
    __device__ __forceinline__ bool next(WsLoad& L)
    {
        const int64_t tk = atomicAdd(ticket, 1);
        if (tk >= total) return false;
        const FrogItem it = items[tk];
        const bool hv = sl.v0 != nullptr;
        L.na = it.na;
        L.nb = it.nb;
        const int64_t ra = it.na > 0 ? it.ra : 0, rb = it.nb > 0 ? it.rb : 0;
        L.plain_a = it.na > 0 && ra < sl.n && ra + it.na > sl.n;
        L.plain_b = it.nb > 0 && rb < sl.n && rb + it.nb > sl.n;
        L.slot_a = ra;
        L.slot_b = rb;
        L.ak = sl.kp(ra); L.av = hv ? sl.vp(ra) : nullptr;
        L.bk = sl.kp(rb); L.bv = hv ? sl.vp(rb) : nullptr;
        L.ak_end = ra < sl.n ? sl.k0 + sl.n : sl.k1 + sl.b;
        L.av_end = hv ? (ra < sl.n ? sl.v0 + sl.n : sl.v1 + sl.b) : nullptr;
        L.bk_end = rb < sl.n ? sl.k0 + sl.n : sl.k1 + sl.b;
        L.bv_end = hv ? (rb < sl.n ? sl.v0 + sl.n : sl.v1 + sl.b) : nullptr;
        const int64_t o = it.oslot, cnt = (int64_t)it.na + it.nb;
        const bool contiguous = (o + cnt <= sl.n) || (o >= sl.n);
        L.dk = contiguous ? sl.kp(o) : nullptr;
        L.dv = contiguous && hv ? sl.vp(o) : nullptr;
        L.oslot = o;
        L.decode = decode;
        L.tk = it.id;                 // the item's flag (node-major id)
        L.dep_lo = it.dep_lo;
        L.dep_hi = it.dep_hi;
        L.flags = it.flags;
        return true;
    }
};

template <int S>
__global__ void __launch_bounds__(WS_CONSUMERS + 32, ws_ctas_per_sm<S>())
    merge_pass_ws_kernel(const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sv, uint64_t* __restrict__ dk,
                         uint32_t* __restrict__ dv, int64_t n, int64_t w, int64_t nblocks,
                         const int64_t* __restrict__ splits, int mode, int decode_out, int* call_err,
                         uint64_t limit_ns, const int* presorted)
{
    if (skip_all(presorted) || (int64_t)blockIdx.x >= nblocks) return;
    PlainLevelSrc<WS_CHUNK> src{sk, sv, dk, dv, n, w, nblocks, splits, decode_out, (int64_t)blockIdx.x};
    ws_merge_out<WS_CONSUMERS, WS_ITEMS, S>(src, sv != nullptr, mode, call_err, limit_ns);
}

// SYM: the symmetric variants' levels (nodes of either orientation).
template <int S, bool SYM = false>
__global__ void __launch_bounds__(WS_CONSUMERS + 32, ws_frog_ctas_per_sm<S>())
    frog_merge_ws_kernel(Slots sl, const FrogItem* __restrict__ items, int64_t total, int mode, int decode_out,
                         int* ticket, int* loaded, int epoch, int* call_err, uint64_t limit_ns, int64_t skip_ticket,
                         const int* presorted, uint32_t jitter_ns)
{
    if (skip_all(presorted)) return;
    FrogLevelSrc src{sl, items, total, ticket, decode_out};
    ws_merge<WS_CONSUMERS, WS_ITEMS, S, true, SYM>(src, sl, sl.v0 != nullptr, mode, call_err, limit_ns, loaded,
                                                   epoch, skip_ticket, jitter_ns);
}

}  // namespace gns
