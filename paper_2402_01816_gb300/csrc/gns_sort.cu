// gns_sort.cu -- host orchestration of the plain stable mergesort (both tiers).
//
// Pass schedule for n > TILE:
//   run detection (1 read pass; early exit for presorted / strictly reversed)
//   100% tier : tile sort -> ceil(log2(n / TILE)) Nocopy merge levels, the tile
//               sort writing to the buffer when the level count is odd so that
//               the last level lands in the caller's arrays ("Forgotten art").
//   50% tier  : node plan -> fused setup (tile sort + scatter into the gapped
//               Frogsort1 leaf slots) -> one in-place merge level per tree depth
//               ("Symmetric merging", "Frogsort1").
//   < 50% tier: the same with Frogsort2's imbalanced tree (inner fraction p =
//               buffer_fraction, floor(p n) buffer; "Frogsort2"), planned on the
//               host: nodes of very different sizes share a depth, so each
//               depth gets its own node list and chunk numbering.
// Keys are encoded (order map) when first read and decoded by the last write.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "gns_internal.h"
#include "gns_kernels.cuh"
#include "gns_merge_tma.cuh"
#include "gns_merge_ws.cuh"

namespace gns {

namespace {

constexpr size_t kSmemTile = sizeof(SmemKV<TILE>);
template <int S>
constexpr size_t ws_smem() { return sizeof(WsSmem<WS_CHUNK, S>); }
template <int S>
constexpr size_t ws_smem_out() { return sizeof(WsSmemOut<WS_CHUNK, S>); }

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }

// Merge levels of the 100% tier: ceil(log2(#tiles)).
int merge_levels(int64_t n)
{
    int64_t tiles = ceil_div(n, TILE);
    int L = 0;
    while ((1ll << L) < tiles) ++L;
    return L;
}

// Leaf depth of the Frogsort1 tree: the first depth whose nodes hold <= TILE
// elements (node sizes at depth d are floor or ceil of n / 2^d).
int frog_leaf_depth(int64_t n)
{
    int D = 0;
    while (ceil_div(n, 1ll << D) > TILE) ++D;
    return D;
}

int64_t frog_chunks(int64_t n, int d) { return ceil_div(ceil_div(n, 1ll << d), CHUNK); }

// Frogsort2 inner fraction p = pn / FROG2_DEN for buffer_fraction < 1/2.
constexpr int64_t FROG2_DEN = 1 << 16;
int64_t frog2_num(double bf) { return (int64_t)(bf * (double)FROG2_DEN + 0.5); }

// Frogsort2 split (Frogsort2 section): the inner child gets floor(p n) elements,
// the outer child floor(p n_outer) buffer slots and the inner child the rest of
// the node's buffer, so every node keeps at least floor(p n) = n_inner slots.
void frog2_split(const FrogNode& p, int64_t pn, FrogNode& L, FrogNode& R)
{
    const int64_t n_inner = p.n * pn / FROG2_DEN, n_outer = p.n - n_inner;
    const int64_t b_outer = n_outer * pn / FROG2_DEN, b_inner = p.b - b_outer;
    if (p.side == 0) { L.n = n_outer; L.b = b_outer; R.n = n_inner; R.b = b_inner; }
    else             { L.n = n_inner; L.b = b_inner; R.n = n_outer; R.b = b_outer; }
    L.side = 0; R.side = 1; L.ori = R.ori = 0;
    L.r = p.r; R.r = p.r + L.n + L.b;
    L.s = p.s; R.s = p.s + L.n;
}

// The Frogsort2 tree, depth by depth (nodes of at most TILE elements are
// leaves, sorted at setup).  Depth d's internal nodes are
// internal[first_node[d], first_node[d+1]), their children pairs follow the
// same order in `children`, and their chunks are numbered by
// cstart[first_cs[d] + k] (k-th node of the depth) up to cstart[first_cs[d] + nk].
struct Frog2Plan {
    std::vector<FrogNode> internal, children, leaves;
    std::vector<int64_t> cstart, first_node, first_cs;
    // Ticket order of each depth, interleaved across its nodes (frog_items_kernel):
    // round j hands out chunk position j of every node holding more than j
    // chunks.  Each depth's nodes are listed largest first, so the nodes of a
    // round are a prefix of the list; iseg holds, from first_sg[d] on, triples
    // (first ticket, first round, nodes per round) of the runs of rounds with
    // one node count.
    std::vector<int32_t> iseg;
    std::vector<int64_t> first_sg;
    // index into `leaves` of the outermost leaf of internal[i] (i < #internal)
    // and of children[j] (at #internal + j): a node of a symmetric variant
    // takes that leaf's orientation (frog_orient_kernel)
    std::vector<int32_t> outer_leaf;
    int64_t max_items = 0;
    int D = 0;
};

Frog2Plan frog2_plan(int64_t n, int64_t pn)
{
    Frog2Plan P;
    std::vector<FrogNode> cur(1), nxt;
    cur[0].n = n; cur[0].b = n * pn / FROG2_DEN; cur[0].r = 0; cur[0].s = 0; cur[0].side = 0; cur[0].ori = 0;
    while (!cur.empty()) {
        nxt.clear();
        // largest first: the interleaved ticket order takes a prefix of the list
        std::stable_sort(cur.begin(), cur.end(), [](const FrogNode& a, const FrogNode& b) { return a.n > b.n; });
        const int64_t first = (int64_t)P.internal.size(), first_c = (int64_t)P.cstart.size();
        int64_t acc = 0;
        for (const FrogNode& x : cur) {
            if (x.n <= TILE) {
                P.leaves.push_back(x);
                continue;
            }
            FrogNode L, R;
            frog2_split(x, pn, L, R);
            P.internal.push_back(x);
            P.children.push_back(L);
            P.children.push_back(R);
            P.cstart.push_back(acc);
            acc += ceil_div(x.n, CHUNK);
            nxt.push_back(L);
            nxt.push_back(R);
        }
        if ((int64_t)P.internal.size() == first) break;
        P.cstart.push_back(acc);
        {
            const int64_t nk = (int64_t)P.internal.size() - first;
            auto chunks = [&](int64_t k) { return P.cstart[first_c + k + 1] - P.cstart[first_c + k]; };
            P.first_sg.push_back((int64_t)P.iseg.size() / 3);
            // rounds [v, v') with v, v' consecutive distinct chunk counts (from 0
            // up) have the same nodes: those whose count reaches v'
            int64_t ts = 0, v = 0;
            for (int64_t i = nk - 1; i >= 0; --i) {
                const int64_t m = chunks(i);
                if (m <= v) continue;
                const int64_t cnt = i + 1;              // nodes with count >= m (listed largest first)
                P.iseg.push_back((int32_t)ts);         // a depth has fewer than 2^31 chunks
                P.iseg.push_back((int32_t)v);
                P.iseg.push_back((int32_t)cnt);
                ts += cnt * (m - v);
                v = m;
            }
        }
        P.first_node.push_back(first);
        P.first_cs.push_back(first_c);
        P.max_items = acc > P.max_items ? acc : P.max_items;
        ++P.D;
        cur.swap(nxt);
    }
    P.first_node.push_back((int64_t)P.internal.size());
    P.first_sg.push_back((int64_t)P.iseg.size() / 3);
    std::sort(P.leaves.begin(), P.leaves.end(), [](const FrogNode& a, const FrogNode& b) { return a.s < b.s; });
    // outermost leaf: a data-left node's leftmost leaf (the one starting at its
    // first element), a data-right node's rightmost (the one holding its last)
    auto leaf_at = [&](int64_t pos) {
        int64_t lo = 0, hi = (int64_t)P.leaves.size() - 1;    // last leaf with s <= pos
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (P.leaves[mid].s <= pos) lo = mid;
            else hi = mid - 1;
        }
        return (int32_t)lo;
    };
    for (const std::vector<FrogNode>* v : {&P.internal, &P.children})
        for (const FrogNode& x : *v) P.outer_leaf.push_back(leaf_at(x.side == 0 ? x.s : x.s + x.n - 1));
    return P;
}

// Frogsort2 plans, uploaded once per (device, n, p) and kept: the host work
// (building the tree) and the upload would otherwise idle the GPU on every
// call.  A handful of shapes are kept; an evicted plan's device copy is freed
// after the device has finished every call that may still read it.
struct Frog2Dev {
    int dev = -1;
    int64_t n = 0, pn = 0;
    Frog2Plan plan;               // host copy: per-depth offsets and totals
    char* d = nullptr;            // internal | children | leaves | cstart | iseg | outer_leaf
    size_t o_ch = 0, o_lv = 0, o_cs = 0, o_sg = 0, o_ol = 0;
    uint64_t used = 0;
};
std::mutex g_frog2_mu;
std::vector<Frog2Dev> g_frog2;
uint64_t g_frog2_clock = 0;
constexpr size_t kFrog2Cache = 4;

// Returns the cached plan for (current device, n, pn), uploading it if new;
// nullptr on a CUDA error.  The caller holds g_frog2_mu.
const Frog2Dev* frog2_get(int64_t n, int64_t pn)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    for (Frog2Dev& e : g_frog2)
        if (e.dev == dev && e.n == n && e.pn == pn) {
            e.used = ++g_frog2_clock;
            return &e;
        }
    Frog2Dev e;
    e.dev = dev; e.n = n; e.pn = pn;
    e.plan = frog2_plan(n, pn);
    const Frog2Plan& P = e.plan;
    e.o_ch = P.internal.size() * sizeof(FrogNode);
    e.o_lv = e.o_ch + P.children.size() * sizeof(FrogNode);
    e.o_cs = e.o_lv + P.leaves.size() * sizeof(FrogNode);
    e.o_sg = e.o_cs + P.cstart.size() * sizeof(int64_t);
    e.o_ol = e.o_sg + P.iseg.size() * sizeof(int32_t);
    const size_t bytes = e.o_ol + P.outer_leaf.size() * sizeof(int32_t);
    std::vector<char> blob(bytes);
    if (!P.internal.empty()) memcpy(blob.data(), P.internal.data(), e.o_ch);
    if (!P.children.empty()) memcpy(blob.data() + e.o_ch, P.children.data(), e.o_lv - e.o_ch);
    if (!P.leaves.empty()) memcpy(blob.data() + e.o_lv, P.leaves.data(), e.o_cs - e.o_lv);
    if (!P.cstart.empty()) memcpy(blob.data() + e.o_cs, P.cstart.data(), e.o_sg - e.o_cs);
    if (!P.iseg.empty()) memcpy(blob.data() + e.o_sg, P.iseg.data(), e.o_ol - e.o_sg);
    if (!P.outer_leaf.empty()) memcpy(blob.data() + e.o_ol, P.outer_leaf.data(), bytes - e.o_ol);
    if (cudaMalloc(&e.d, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaMemcpy(e.d, blob.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(e.d);
        return nullptr;
    }
    e.used = ++g_frog2_clock;
    if (g_frog2.size() >= kFrog2Cache) {
        size_t v = 0;
        for (size_t i = 1; i < g_frog2.size(); ++i)
            if (g_frog2[i].used < g_frog2[v].used) v = i;
        int cur = dev;
        cudaSetDevice(g_frog2[v].dev);
        cudaDeviceSynchronize();                     // no call still reads the evicted plan
        cudaFree(g_frog2[v].d);
        cudaSetDevice(cur);
        g_frog2.erase(g_frog2.begin() + (long)v);
    }
    g_frog2.push_back(std::move(e));
    return &g_frog2.back();
}

struct Layout {
    // control words (ints): [0..1] presorted flags, [2] call error
    size_t ctl, bufk, bufv, splits, items, nodes, flags, tickets, leaf_ori, total;
    size_t flags_bytes, tickets_bytes;
    int L, D;
};

// sym: a symmetric variant (per-call copies of a host-planned tree's nodes).
Layout make_layout(int64_t n, double bf, bool with_vals, const Frog2Plan* plan, bool sym = false)
{
    Layout o{};
    size_t off = 0;
    o.ctl = off; off += 256;
    if (n <= TILE) { o.total = off; return o; }
    if (bf < 0.5 && plan) {
        const int64_t b = n * frog2_num(bf) / FROG2_DEN;
        o.D = plan->D;
        o.bufk = off; off += align256((size_t)b * 8);
        o.bufv = off; off += with_vals ? align256((size_t)b * 4) : 0;
        o.splits = off; off += align256((size_t)plan->max_items * 8);
        o.items = off; off += align256((size_t)plan->max_items * sizeof(FrogItem));
        o.flags = off; o.flags_bytes = align256((plan->leaves.size() + (size_t)plan->max_items) * 4);
        off += o.flags_bytes;
        o.tickets = off; o.tickets_bytes = align256((size_t)(plan->D + 2) * 4); off += o.tickets_bytes;
        if (sym) {
            // the leaves' orientations and a copy of the internal and child
            // nodes, whose orientations are set per call
            o.leaf_ori = off; off += align256(plan->leaves.size() * 4);
            o.nodes = off; off += align256((plan->internal.size() + plan->children.size()) * sizeof(FrogNode));
        }
    } else if (bf >= 1.0) {
        o.L = merge_levels(n);
        int64_t nblocks = ceil_div(n, CHUNK);
        o.bufk = off; off += align256((size_t)n * 8);
        o.bufv = off; off += with_vals ? align256((size_t)n * 4) : 0;
        o.splits = off; off += align256((size_t)nblocks * 8);
    } else {
        int D = frog_leaf_depth(n);
        o.D = D;
        int64_t b = n / 2;
        o.bufk = off; off += align256((size_t)b * 8);
        o.bufv = off; off += with_vals ? align256((size_t)b * 4) : 0;
        o.nodes = off; off += align256((size_t)((2ll << D) - 1) * sizeof(FrogNode));
        int64_t max_split = 0;
        for (int d = 0; d < D; ++d) {
            int64_t e = (1ll << d) * frog_chunks(n, d);
            if (e > max_split) max_split = e;
        }
        const int64_t nflags = (1ll << D) + max_split;   // one per leaf (setup), one per ticket (all levels)
        o.splits = off; off += align256((size_t)max_split * 8);
        o.items = off; off += align256((size_t)max_split * sizeof(FrogItem));
        o.flags = off; o.flags_bytes = align256((size_t)nflags * 4); off += o.flags_bytes;
        o.tickets = off; o.tickets_bytes = align256((size_t)(D + 1) * 4); off += o.tickets_bytes;
        o.leaf_ori = off; off += align256((size_t)(1ll << D) * 4);   // symmetric variants
    }
    o.total = off;
    return o;
}

template <typename K>
void set_smem(K kernel, size_t bytes)
{
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

PerDeviceOnce g_attr_once;

void init_attributes()
{
    g_attr_once.run([] {
        set_smem(tile_sort_kernel<SORT_THREADS, SORT_ITEMS>, kSmemTile);
        set_smem(frog_setup_kernel<SORT_THREADS, SORT_ITEMS, FROG_PLAIN>, kSmemTile);
        set_smem(frog_setup_kernel<SORT_THREADS, SORT_ITEMS, FROG_GECKO>, kSmemTile);
        set_smem(frog_setup_kernel<SORT_THREADS, SORT_ITEMS, FROG_SQUID>, kSmemTile);
        set_smem(merge_pass_ws_kernel<2>, ws_smem_out<2>());
        set_smem(merge_pass_ws_kernel<3>, ws_smem_out<3>());
        set_smem(merge_pass_ws_kernel<4>, ws_smem_out<4>());
        set_smem(frog_merge_ws_kernel<2>, ws_smem<2>());
        set_smem(frog_merge_ws_kernel<3>, ws_smem<3>());
        set_smem(frog_merge_ws_kernel<4>, ws_smem<4>());
        set_smem(frog_merge_ws_kernel<2, true>, ws_smem<2>());
        set_smem(frog_merge_ws_kernel<3, true>, ws_smem<3>());
        set_smem(frog_merge_ws_kernel<4, true>, ws_smem<4>());
    });
}

// Merge-level pipeline (GNS_MERGE_PIPE overrides the default):
//   "ws2", "ws3", "ws4"  warp-specialised with 2 / 3 / 4 stages
//   (gns_merge_ws.cuh).  The 100% levels default to ws2: with their out
//   buffer that is the most resident CTAs, measured fastest; storing each
//   chunk from its own input stage instead (no out buffer, three 3-stage CTAs
//   per SM) measured 2% slower per level.
enum MergePipe { PIPE_WS2 = 0, PIPE_WS3, PIPE_WS4 };

int pipe_from_env(const char* name, int dflt)
{
    const char* e = getenv(name);
    if (!e) return dflt;
    if (!strcmp(e, "ws2")) return (int)PIPE_WS2;
    if (!strcmp(e, "ws3")) return (int)PIPE_WS3;
    if (!strcmp(e, "ws4")) return (int)PIPE_WS4;
    return dflt;
}

int merge_pipe()
{
    static const int v = pipe_from_env("GNS_MERGE_PIPE", PIPE_WS2);
    return v;
}

// The in-place levels' pipeline (GNS_FROG_PIPE; default ws3: three 3-stage
// CTAs per SM, measured 3% faster per level than ws2 at 2^27).
int frog_pipe()
{
    static const int v = pipe_from_env("GNS_FROG_PIPE", PIPE_WS3);
    return v;
}

// Resident CTAs of a kernel at its launch shape, over all SMs.
template <typename K>
int64_t resident_ctas(K kernel, int threads, size_t smem)
{
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, smem) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        v = 1;
    }
    return (int64_t)v * num_sms();
}

// Resident CTAs of a kernel at its launch shape on the current device, looked
// up once per device.
template <typename K>
int64_t resident_ctas_cached(int64_t (&cache)[64], K kernel, int threads, size_t smem)
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return resident_ctas(kernel, threads, smem);
    if (!cache[dev]) cache[dev] = resident_ctas(kernel, threads, smem);
    return cache[dev];
}

template <int S>
cudaError_t launch_plain_level_ws(const uint64_t* sk, const uint32_t* sv, uint64_t* dk, uint32_t* dv, int64_t n,
                                  int64_t w, int64_t nblocks, const int64_t* splits, int mode, int decode,
                                  int* call_err, uint64_t limit, const int* skip, cudaStream_t s)
{
    static int64_t caps[64] = {};
    const int64_t cap = resident_ctas_cached(caps, merge_pass_ws_kernel<S>, WS_CONSUMERS + 32, ws_smem_out<S>());
    const int64_t grid = imin(nblocks, cap);
    return launch(K_MERGE_PASS, merge_pass_ws_kernel<S>, dim3((unsigned)grid), dim3(WS_CONSUMERS + 32),
                  ws_smem_out<S>(), s, sk, sv, dk, dv, n, w, nblocks, splits, mode, decode, call_err, limit, skip);
}

template <int S, bool SYM>
cudaError_t launch_frog_level_ws(const Slots& sl, const FrogItem* items, int64_t total, int mode, int decode,
                                 int* ticket, int* loaded, int epoch, int* call_err, uint64_t limit,
                                 int64_t skip_ticket, const int* skip, cudaStream_t s)
{
    static int64_t caps[64] = {};
    const int64_t cap =
        resident_ctas_cached(caps, frog_merge_ws_kernel<S, SYM>, WS_CONSUMERS + 32, ws_smem<S>());
    const int64_t grid = imin(total, cap);
    return launch(K_FROG_MERGE, frog_merge_ws_kernel<S, SYM>, dim3((unsigned)grid), dim3(WS_CONSUMERS + 32),
                  ws_smem<S>(), s, sl, items, total, mode, decode, ticket, loaded, epoch, call_err, limit,
                  skip_ticket, skip, debug_jitter_ns());
}

cudaError_t launch_plain_level(const uint64_t* sk, const uint32_t* sv, uint64_t* dk, uint32_t* dv, int64_t n,
                               int64_t w, int64_t nblocks, const int64_t* splits, int mode, int decode,
                               int* call_err, uint64_t limit, const int* skip, cudaStream_t s)
{
#define GNS_PLAIN_ARGS sk, sv, dk, dv, n, w, nblocks, splits, mode, decode, call_err, limit, skip, s
    switch (merge_pipe()) {
    case PIPE_WS2: return launch_plain_level_ws<2>(GNS_PLAIN_ARGS);
    case PIPE_WS3: return launch_plain_level_ws<3>(GNS_PLAIN_ARGS);
    case PIPE_WS4: return launch_plain_level_ws<4>(GNS_PLAIN_ARGS);
    default: return launch_plain_level_ws<2>(GNS_PLAIN_ARGS);
    }
#undef GNS_PLAIN_ARGS
}

cudaError_t launch_frog_level(const Slots& sl, const FrogItem* items, int64_t total, int mode, int decode,
                              int* ticket, int* loaded, int epoch, int* call_err, uint64_t limit, int64_t skip_ticket,
                              const int* skip, cudaStream_t s, bool sym = false)
{
#define GNS_FROG_ARGS sl, items, total, mode, decode, ticket, loaded, epoch, call_err, limit, skip_ticket, skip, s
    if (sym) {
        switch (frog_pipe()) {
        case PIPE_WS2: return launch_frog_level_ws<2, true>(GNS_FROG_ARGS);
        case PIPE_WS4: return launch_frog_level_ws<4, true>(GNS_FROG_ARGS);
        default: return launch_frog_level_ws<3, true>(GNS_FROG_ARGS);
        }
    }
    switch (frog_pipe()) {
    case PIPE_WS2: return launch_frog_level_ws<2, false>(GNS_FROG_ARGS);
    case PIPE_WS3: return launch_frog_level_ws<3, false>(GNS_FROG_ARGS);
    case PIPE_WS4: return launch_frog_level_ws<4, false>(GNS_FROG_ARGS);
    default: return launch_frog_level_ws<2, false>(GNS_FROG_ARGS);
    }
#undef GNS_FROG_ARGS
}

#define GNS_TRY(x)                              \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) {                \
            rc = GNS_ERR_CUDA;                  \
            goto done;                          \
        }                                       \
    } while (0)

}  // namespace

cudaError_t publish_call_error(const int* call_err, cudaStream_t s)
{
    int* st = status_word_ptr();
    if (!st) return cudaErrorUnknown;
    return launch(K_ERR_PUBLISH, publish_err_kernel, dim3(1), dim3(1), 0, s, call_err, st);
}

size_t sort_workspace_bytes(int64_t n, double bf)
{
    if (n <= 1) return 0;
    if (bf < 0.5 && n > TILE) {
        const Frog2Plan plan = frog2_plan(n, frog2_num(bf));
        // the plan itself is kept by the library (frog2_get), apart from the workspace
        const size_t plan_bytes = (plan.internal.size() + plan.children.size() + plan.leaves.size()) *
                                      sizeof(FrogNode) + plan.cstart.size() * sizeof(int64_t) +
                                  (plan.outer_leaf.size() + plan.iseg.size()) * sizeof(int32_t);
        return make_layout(n, bf, true, &plan).total + align256(plan_bytes);
    }
    return make_layout(n, bf, true, nullptr).total;
}

namespace {

// Run detection (one read pass) and the reversal of strictly descending input;
// ctl must be reset already.
cudaError_t detect_and_reverse(uint64_t* keys, uint32_t* vals, int64_t n, int mode, int* ctl, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(ctl, 1, 2 * sizeof(int), s);   // both flags "true"
    if (e != cudaSuccess) return e;
    // one wave of persistent CTAs: a second partial wave would start its tiles late
    static int64_t caps[64] = {};
    const int64_t detect_cap = resident_ctas_cached(caps, run_detect_kernel, DETECT_THREADS, 0);
    e = launch(K_RUN_DETECT, run_detect_kernel, dim3((unsigned)imin(ceil_div(n, DETECT_TILE), detect_cap)),
               dim3(DETECT_THREADS), 0, s, (const uint64_t*)keys, n, mode, ctl);
    if (e != cudaSuccess) return e;
    return launch(K_REVERSE, reverse_kernel, dim3((unsigned)(num_sms() * 8)), dim3(256), 0, s, keys, vals, n,
                  (const int*)ctl);
}

}  // namespace

int64_t plain_sort_splits(int64_t n) { return n > TILE ? ceil_div(n, CHUNK) : 0; }

int plain_sort_ext(uint64_t* keys, uint32_t* vals, int64_t n, int mode, uint64_t* bufk, uint32_t* bufv,
                   int64_t* splits, int* ctl, const int* gate, cudaStream_t s)
{
    if (n <= 1) return GNS_OK;
    init_attributes();
    int rc = GNS_OK;
    int* call_err = ctl + 2;
    const int* skip = ctl;
    const int L = merge_levels(n);
    uint64_t* cur_k = (L & 1) ? bufk : keys;
    uint32_t* cur_v = (L & 1) ? bufv : vals;
    uint64_t* oth_k = (L & 1) ? keys : bufk;
    uint32_t* oth_v = (L & 1) ? vals : bufv;
    if (!vals) cur_v = oth_v = nullptr;
    const int64_t nblocks = ceil_div(n, CHUNK);
    GNS_TRY(cudaMemsetAsync(ctl, 0, 256, s));
    if (gate)
        GNS_TRY(launch(K_RUN_DETECT, gate_kernel, dim3(1), dim3(1), 0, s, gate, ctl));
    else
        GNS_TRY(detect_and_reverse(keys, vals, n, mode, ctl, s));
    // the tile sort writes to the buffer when the level count is odd, so that
    // the last level lands in the caller's arrays; with no level it decodes
    GNS_TRY(launch(K_TILE_SORT, tile_sort_kernel<SORT_THREADS, SORT_ITEMS>, dim3((unsigned)ceil_div(n, TILE)),
                   dim3(SORT_THREADS), kSmemTile, s, (const uint64_t*)keys, (const uint32_t*)vals, cur_k, cur_v, n,
                   mode, (int)(L == 0), skip));
    for (int lvl = 0; lvl < L; ++lvl) {
        const int64_t w = (int64_t)TILE << lvl;
        GNS_TRY(launch(K_MERGE_PARTITION, merge_partition_kernel, dim3((unsigned)ceil_div(nblocks, 256)), dim3(256),
                       0, s, (const uint64_t*)cur_k, n, w, nblocks, splits, skip));
        GNS_TRY(launch_plain_level((const uint64_t*)cur_k, (const uint32_t*)cur_v, oth_k, oth_v, n, w, nblocks,
                                   (const int64_t*)splits, mode, (int)(lvl == L - 1), call_err, wait_limit_ns(), skip,
                                   s));
        uint64_t* tk = cur_k; cur_k = oth_k; oth_k = tk;
        uint32_t* tv = cur_v; cur_v = oth_v; oth_v = tv;
    }
    GNS_TRY(publish_call_error(call_err, s));
done:
    return rc;
}

// variant (the in-place tiers, bf < 1): FROG_PLAIN = Frogsort1/2, FROG_GECKO =
// Geckosort, FROG_SQUID = Squidsort (frog_setup_kernel), on Frogsort1's tree
// for bf in [0.5, 1) and on Frogsort2's below.
int sort_device_variant(uint64_t* keys, uint32_t* vals, int64_t n, int mode, double bf, int variant,
                        cudaStream_t s)
{
    if (n <= 1) return GNS_OK;
    if (bf >= 1.0 || n <= TILE) {
        const Layout lay = make_layout(n, 1.0, vals != nullptr, nullptr);
        char* ws = (char*)ws_alloc(lay.total, s);
        if (!ws) return GNS_ERR_OOM;
        const int rc = plain_sort_ext(keys, vals, n, mode, n > TILE ? (uint64_t*)(ws + lay.bufk) : nullptr,
                                      (vals && n > TILE) ? (uint32_t*)(ws + lay.bufv) : nullptr,
                                      n > TILE ? (int64_t*)(ws + lay.splits) : nullptr, (int*)(ws + lay.ctl),
                                      nullptr, s);
        ws_free(ws, s);
        return rc;
    }
    const bool frog2 = bf < 0.5;
    std::unique_lock<std::mutex> plan_lock(g_frog2_mu, std::defer_lock);
    const Frog2Dev* fp = nullptr;
    if (frog2) {
        plan_lock.lock();                            // held for the call: the entry may not be evicted
        fp = frog2_get(n, frog2_num(bf));
        if (!fp) return GNS_ERR_CUDA;
    }
    const Layout lay = make_layout(n, bf, vals != nullptr, frog2 ? &fp->plan : nullptr, variant != FROG_PLAIN);
    char* ws = (char*)ws_alloc(lay.total, s);
    if (!ws) return GNS_ERR_OOM;
    init_attributes();
    int rc = GNS_OK;
    int* ctl = (int*)(ws + lay.ctl);
    int* call_err = ctl + 2;
    const int* skip = ctl;

    GNS_TRY(cudaMemsetAsync(ctl, 0, 256, s));
    GNS_TRY(detect_and_reverse(keys, vals, n, mode, ctl, s));

    if (frog2) {
        const int D = lay.D;
        Slots sl;
        sl.k0 = keys; sl.v0 = vals; sl.n = n; sl.b = n * frog2_num(bf) / FROG2_DEN;
        sl.k1 = (uint64_t*)(ws + lay.bufk);
        sl.v1 = vals ? (uint32_t*)(ws + lay.bufv) : nullptr;
        const Frog2Plan& plan = fp->plan;
        const bool sym = variant != FROG_PLAIN;
        // symmetric variants: the node lists are copied per call, since the
        // data sets their orientations (the cached plan is shared)
        const int64_t nlist = (int64_t)(plan.internal.size() + plan.children.size());
        FrogNode* nodes2 = (FrogNode*)(ws + lay.nodes);
        int* leaf_ori = (int*)(ws + lay.leaf_ori);
        if (sym) GNS_TRY(cudaMemcpyAsync(nodes2, fp->d, (size_t)nlist * sizeof(FrogNode), cudaMemcpyDeviceToDevice, s));
        const FrogNode* internal = sym ? nodes2 : (const FrogNode*)fp->d;
        const FrogNode* children = sym ? nodes2 + plan.internal.size() : (const FrogNode*)(fp->d + fp->o_ch);
        const FrogNode* leaves = (const FrogNode*)(fp->d + fp->o_lv);
        const int64_t* cstart = (const int64_t*)(fp->d + fp->o_cs);
        int64_t* splits = (int64_t*)(ws + lay.splits);
        FrogItem* items = (FrogItem*)(ws + lay.items);
        int* flags = (int*)(ws + lay.flags);
        int* tickets = (int*)(ws + lay.tickets);
        const uint64_t limit = wait_limit_ns();
        GNS_TRY(cudaMemsetAsync(flags, 0, lay.flags_bytes + lay.tickets_bytes, s));
        const int64_t nleaves = (int64_t)plan.leaves.size();
        const dim3 sgrid((unsigned)nleaves), sblock(SORT_THREADS);
#define GNS_SETUP2_ARGS sl, leaves, nleaves, mode, tickets + D, flags, call_err, limit, skip, leaf_ori, debug_jitter_ns()
        if (variant == FROG_GECKO)
            GNS_TRY(launch(K_FROG_SETUP, frog_setup_kernel<SORT_THREADS, SORT_ITEMS, FROG_GECKO>, sgrid, sblock,
                           kSmemTile, s, GNS_SETUP2_ARGS));
        else if (variant == FROG_SQUID)
            GNS_TRY(launch(K_FROG_SETUP, frog_setup_kernel<SORT_THREADS, SORT_ITEMS, FROG_SQUID>, sgrid, sblock,
                           kSmemTile, s, GNS_SETUP2_ARGS));
        else
            GNS_TRY(launch(K_FROG_SETUP, frog_setup_kernel<SORT_THREADS, SORT_ITEMS, FROG_PLAIN>, sgrid, sblock,
                           kSmemTile, s, GNS_SETUP2_ARGS));
#undef GNS_SETUP2_ARGS
        if (sym && nlist > 0)
            GNS_TRY(launch(K_FROG_PLAN, frog_orient_list_kernel, dim3((unsigned)ceil_div(nlist, 256)), dim3(256), 0, s,
                           nodes2, nlist, (const int32_t*)(fp->d + fp->o_ol), (const int*)leaf_ori, skip));
        int* lflags = flags + nleaves;
        int64_t skip_ticket = take_debug_skip_publish();
        for (int d = D - 1; d >= 0; --d) {
            const int64_t f0 = plan.first_node[d], nnodes = plan.first_node[d + 1] - f0;
            const int64_t c0 = plan.first_cs[d], total = plan.cstart[c0 + nnodes];
            const FrogNode* level = internal + f0;
            const FrogNode* child = children + 2 * f0;
            const int64_t* cs = cstart + c0;
            const int32_t* sg = (const int32_t*)(fp->d + fp->o_sg) + 3 * plan.first_sg[d];
            const int64_t nsg = plan.first_sg[d + 1] - plan.first_sg[d];
            const dim3 pgrid((unsigned)ceil_div(total, 256));
            if (sym) {
                GNS_TRY(launch(K_FROG_PARTITION, frog_partition_kernel<true>, pgrid, dim3(256), 0, s, sl, level,
                               child, nnodes, (int64_t)0, cs, total, splits, skip));
                GNS_TRY(launch(K_FROG_PARTITION, frog_items_kernel<true>, pgrid, dim3(256), 0, s, level, child,
                               nnodes, (int64_t)0, cs, total, (const int64_t*)splits, items, call_err, skip,
                               (int)(d != 0), sg, nsg));
            } else {
                GNS_TRY(launch(K_FROG_PARTITION, frog_partition_kernel<false>, pgrid, dim3(256), 0, s, sl, level,
                               child, nnodes, (int64_t)0, cs, total, splits, skip));
                GNS_TRY(launch(K_FROG_PARTITION, frog_items_kernel<false>, pgrid, dim3(256), 0, s, level, child,
                               nnodes, (int64_t)0, cs, total, (const int64_t*)splits, items, call_err, skip,
                               (int)(d != 0), sg, nsg));
            }
            GNS_TRY(launch_frog_level(sl, (const FrogItem*)items, total, mode, (int)(d == 0), tickets + d, lflags,
                                      D - d, call_err, limit, skip_ticket, skip, s, sym));
            skip_ticket = -1;
        }
        if (variant == FROG_SQUID && !plan.internal.empty())   // a mirrored root: the one final reversal
            GNS_TRY(launch(K_REVERSE, reverse_root_kernel, dim3((unsigned)(num_sms() * 8)), dim3(256), 0, s, keys,
                           vals, n, internal, (const int*)ctl));
    } else {
        const int D = lay.D;
        Slots sl;
        sl.k0 = keys; sl.v0 = vals; sl.n = n; sl.b = n / 2;
        sl.k1 = (uint64_t*)(ws + lay.bufk);
        sl.v1 = vals ? (uint32_t*)(ws + lay.bufv) : nullptr;
        FrogNode* nodes = (FrogNode*)(ws + lay.nodes);
        int64_t* splits = (int64_t*)(ws + lay.splits);
        FrogItem* items = (FrogItem*)(ws + lay.items);
        int* flags = (int*)(ws + lay.flags);
        int* tickets = (int*)(ws + lay.tickets);
        const uint64_t limit = wait_limit_ns();
        GNS_TRY(cudaMemsetAsync(flags, 0, lay.flags_bytes + lay.tickets_bytes, s));
        const int64_t total_nodes = (2ll << D) - 1;
        GNS_TRY(launch(K_FROG_PLAN, frog_plan_kernel, dim3((unsigned)ceil_div(total_nodes, 256)), dim3(256), 0, s,
                       nodes, n, D));
        const int64_t nleaves = 1ll << D;
        const FrogNode* leaves = nodes + (nleaves - 1);
        int* leaf_ori = (int*)(ws + lay.leaf_ori);
        const bool sym = variant != FROG_PLAIN;
        const dim3 sgrid((unsigned)nleaves), sblock(SORT_THREADS);
#define GNS_SETUP_ARGS sl, leaves, nleaves, mode, tickets + D, flags, call_err, limit, skip, leaf_ori, debug_jitter_ns()
        if (variant == FROG_GECKO)
            GNS_TRY(launch(K_FROG_SETUP, frog_setup_kernel<SORT_THREADS, SORT_ITEMS, FROG_GECKO>, sgrid, sblock,
                           kSmemTile, s, GNS_SETUP_ARGS));
        else if (variant == FROG_SQUID)
            GNS_TRY(launch(K_FROG_SETUP, frog_setup_kernel<SORT_THREADS, SORT_ITEMS, FROG_SQUID>, sgrid, sblock,
                           kSmemTile, s, GNS_SETUP_ARGS));
        else
            GNS_TRY(launch(K_FROG_SETUP, frog_setup_kernel<SORT_THREADS, SORT_ITEMS, FROG_PLAIN>, sgrid, sblock,
                           kSmemTile, s, GNS_SETUP_ARGS));
#undef GNS_SETUP_ARGS
        if (sym)
            GNS_TRY(launch(K_FROG_PLAN, frog_orient_kernel, dim3((unsigned)ceil_div(total_nodes, 256)), dim3(256), 0,
                           s, nodes, D, (const int*)leaf_ori, skip));
        int* lflags = flags + nleaves;
        int64_t skip_ticket = take_debug_skip_publish();
        for (int d = D - 1; d >= 0; --d) {
            const int64_t nnodes = 1ll << d;
            const int64_t nch = frog_chunks(n, d);
            const FrogNode* level = nodes + (nnodes - 1);
            const FrogNode* child = nodes + (2 * nnodes - 1);
            const dim3 pgrid((unsigned)ceil_div(nnodes * nch, 256));
            if (sym) {
                GNS_TRY(launch(K_FROG_PARTITION, frog_partition_kernel<true>, pgrid, dim3(256), 0, s, sl, level,
                               child, nnodes, nch, (const int64_t*)nullptr, nnodes * nch, splits, skip));
                GNS_TRY(launch(K_FROG_PARTITION, frog_items_kernel<true>, pgrid, dim3(256), 0, s, level, child,
                               nnodes, nch, (const int64_t*)nullptr, nnodes * nch, (const int64_t*)splits, items,
                               call_err, skip, (int)(d != 0), (const int32_t*)nullptr,
                               (int64_t)0));
            } else {
                GNS_TRY(launch(K_FROG_PARTITION, frog_partition_kernel<false>, pgrid, dim3(256), 0, s, sl, level,
                               child, nnodes, nch, (const int64_t*)nullptr, nnodes * nch, splits, skip));
                GNS_TRY(launch(K_FROG_PARTITION, frog_items_kernel<false>, pgrid, dim3(256), 0, s, level, child,
                               nnodes, nch, (const int64_t*)nullptr, nnodes * nch, (const int64_t*)splits, items,
                               call_err, skip, (int)(d != 0), (const int32_t*)nullptr,
                               (int64_t)0));
            }
            GNS_TRY(launch_frog_level(sl, (const FrogItem*)items, nnodes * nch, mode, (int)(d == 0), tickets + d,
                                      lflags, D - d, call_err, limit, skip_ticket, skip, s, sym));
            skip_ticket = -1;
        }
        if (variant == FROG_SQUID)      // a mirrored root: the one final reversal
            GNS_TRY(launch(K_REVERSE, reverse_root_kernel, dim3((unsigned)(num_sms() * 8)), dim3(256), 0, s, keys,
                           vals, n, (const FrogNode*)nodes, (const int*)ctl));
    }
    GNS_TRY(publish_call_error(call_err, s));
done:
    ws_free(ws, s);
    return rc;
}

int sort_device(uint64_t* keys, uint32_t* vals, int64_t n, int mode, double bf, cudaStream_t s)
{
    return sort_device_variant(keys, vals, n, mode, bf, FROG_PLAIN, s);
}

size_t frog_levels_bytes(int64_t n, int D)
{
    int64_t max_split = 1;
    for (int d = 0; d < D; ++d) {
        const int64_t e = (1ll << d) * frog_chunks(n, d);
        if (e > max_split) max_split = e;
    }
    return align256((size_t)max_split * 8) + align256((size_t)max_split * sizeof(FrogItem)) +
           align256((size_t)max_split * 4) + align256((size_t)(D + 1) * 4);
}

int frog_levels_device(const Slots& sl, const FrogNode* nodes, int D, int mode, int* ctl, char* ws, cudaStream_t s)
{
    init_attributes();
    int rc = GNS_OK;
    int64_t max_split = 1;
    for (int d = 0; d < D; ++d) {
        const int64_t e = (1ll << d) * frog_chunks(sl.n, d);
        if (e > max_split) max_split = e;
    }
    int64_t* splits = (int64_t*)ws;
    FrogItem* items = (FrogItem*)(ws + align256((size_t)max_split * 8));
    int* flags = (int*)((char*)items + align256((size_t)max_split * sizeof(FrogItem)));
    int* tickets = (int*)((char*)flags + align256((size_t)max_split * 4));
    int* call_err = ctl + 2;
    const int* skip = ctl;
    const uint64_t limit = wait_limit_ns();
    GNS_TRY(cudaMemsetAsync(flags, 0, align256((size_t)max_split * 4) + align256((size_t)(D + 1) * 4), s));
    for (int d = D - 1; d >= 0; --d) {
        const int64_t nnodes = 1ll << d;
        const int64_t nch = frog_chunks(sl.n, d);
        const FrogNode* level = nodes + (nnodes - 1);
        const FrogNode* child = nodes + (2 * nnodes - 1);
        GNS_TRY(launch(K_FROG_PARTITION, frog_partition_kernel<false>, dim3((unsigned)ceil_div(nnodes * nch, 256)),
                       dim3(256), 0, s, sl, level, child, nnodes, nch, (const int64_t*)nullptr, nnodes * nch, splits,
                       skip));
        GNS_TRY(launch(K_FROG_PARTITION, frog_items_kernel<false>, dim3((unsigned)ceil_div(nnodes * nch, 256)), dim3(256), 0,
                       s, level, child, nnodes, nch, (const int64_t*)nullptr, nnodes * nch, (const int64_t*)splits,
                       items, call_err, skip, (int)(d != 0), (const int32_t*)nullptr, (int64_t)0));
        GNS_TRY(launch_frog_level(sl, (const FrogItem*)items, nnodes * nch, mode, (int)(d == 0), tickets + d, flags,
                                  D - d, call_err, limit, (int64_t)-1, skip, s));
    }
    GNS_TRY(publish_call_error(call_err, s));
done:
    return rc;
}

}  // namespace gns

// ------------------------------------------------------------ plan checks
// Invariants of the trees the in-place tiers run on, checked on the host for a
// test hook (gns_frog_plan_check).  Returns 0, or the number of the first
// invariant that fails:
//   1  children split the parent: sizes and buffers add up, regions adjoin;
//   2  a node holds at least as many buffer slots as its inner child has
//      elements (what the in-place merge needs, "Symmetric merging");
//   3  left children are data-left, right children data-right, input ranges
//      adjoin;
//   4  the leaves, in input order, cover [0, n) without gaps and hold at most
//      one tile each;
//   5  every data slot range lies inside the slots [0, n + b);
//   6  chunk numbering: each depth's node chunks are numbered consecutively;
//   7  ticket order (Frogsort2): each depth's tickets map one to one onto its
//      chunks (frog_items_kernel's mapping from iseg), and within a
//      node the chunk positions come in increasing ticket order.
namespace gns {
namespace {

int check_split(const FrogNode& x, const FrogNode& L, const FrogNode& R, int64_t total)
{
    if (L.n + R.n != x.n || L.b + R.b != x.b || L.r != x.r || R.r != x.r + L.n + L.b) return 1;
    if (L.n < 0 || R.n < 0 || L.b < 0 || R.b < 0) return 1;
    const int64_t inner = x.side == 0 ? R.n : L.n;
    if (x.b < inner) return 2;
    if (L.side != 0 || R.side != 1 || L.s != x.s || R.s != x.s + L.n) return 3;
    for (const FrogNode* c : {&L, &R})
        if (frog_data_slot(*c) < 0 || frog_data_slot(*c) + c->n > total) return 5;
    return 0;
}

int check_leaves(std::vector<FrogNode> leaves, int64_t n, int64_t total)
{
    std::sort(leaves.begin(), leaves.end(), [](const FrogNode& a, const FrogNode& b) { return a.s < b.s; });
    int64_t next = 0;
    for (const FrogNode& x : leaves) {
        if (x.s != next || x.n > TILE) return 4;
        if (frog_data_slot(x) < 0 || frog_data_slot(x) + x.n > total) return 5;
        next += x.n;
    }
    return next == n ? 0 : 4;
}

}  // namespace
}  // namespace gns

extern "C" int gns_frog_plan_check(int64_t n, double buffer_fraction)
{
    using namespace gns;
    if (n <= TILE || !(buffer_fraction > 0.0) || buffer_fraction >= 1.0) return -1;
    if (buffer_fraction < 0.5) {
        const int64_t pn = frog2_num(buffer_fraction);
        const Frog2Plan P = frog2_plan(n, pn);
        const int64_t total = n + n * pn / FROG2_DEN;
        if (P.internal.empty() || P.internal[0].n != n || P.internal[0].r != 0 || P.internal[0].side != 0) return 1;
        for (size_t k = 0; k < P.internal.size(); ++k) {
            const int rc = check_split(P.internal[k], P.children[2 * k], P.children[2 * k + 1], total);
            if (rc) return rc;
        }
        for (int d = 0; d < P.D; ++d) {
            const int64_t f0 = P.first_node[d], nn = P.first_node[d + 1] - f0, c0 = P.first_cs[d];
            if (P.cstart[c0] != 0) return 6;
            for (int64_t k = 0; k < nn; ++k)
                if (P.cstart[c0 + k + 1] - P.cstart[c0 + k] != ceil_div(P.internal[f0 + k].n, CHUNK)) return 6;
            // the device's ticket -> (node, position) mapping, ticket by ticket
            const int64_t tot = P.cstart[c0 + nn], g0 = P.first_sg[d], ns = P.first_sg[d + 1] - g0;
            if (ns < 1) return 7;
            std::vector<char> seen((size_t)tot, 0);
            std::vector<int64_t> next_pos((size_t)nn, 0);
            for (int64_t tk = 0; tk < tot; ++tk) {
                int64_t lo = 0, hi = ns - 1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi + 1) >> 1;
                    if (P.iseg[3 * (g0 + mid)] <= tk) lo = mid;
                    else hi = mid - 1;
                }
                const int64_t off = tk - P.iseg[3 * (g0 + lo)], cnt = P.iseg[3 * (g0 + lo) + 2];
                if (off < 0 || cnt < 1 || cnt > nn) return 7;
                const int64_t local = P.iseg[3 * (g0 + lo) + 1] + off / cnt;
                const int64_t k = off % cnt;
                if (k < 0 || k >= nn) return 7;
                const int64_t base = P.cstart[c0 + k], nchk = P.cstart[c0 + k + 1] - base;
                if (local < 0 || local >= nchk || seen[(size_t)(base + local)]) return 7;
                seen[(size_t)(base + local)] = 1;
                if (local < next_pos[(size_t)k]) return 7;            // positions of a node in ticket order
                next_pos[(size_t)k] = local + 1;
            }
        }
        return check_leaves(P.leaves, n, total);
    }
    // Frogsort1: the node table the plan kernel builds, from the same split
    const int D = frog_leaf_depth(n);
    const int64_t total = n + n / 2;
    std::vector<FrogNode> level(1), next, leaves;
    level[0].n = n; level[0].b = n / 2; level[0].r = 0; level[0].s = 0; level[0].side = 0; level[0].ori = 0;
    for (int d = 0; d < D; ++d) {
        next.clear();
        for (const FrogNode& x : level) {
            FrogNode L, R;
            frog_split(x, L, R);
            const int rc = check_split(x, L, R, total);
            if (rc) return rc;
            if (ceil_div(x.n, CHUNK) > frog_chunks(n, d)) return 6;
            next.push_back(L);
            next.push_back(R);
        }
        level.swap(next);
    }
    return check_leaves(level, n, total);
}

// Test hook: the merge-path partition of one 100%-tier level on its own
// (merge_partition_kernel), so that the co-ranks can be checked against their
// definition.
extern "C" int gns_debug_merge_partition(const uint64_t* keys, int64_t n, int64_t w, int64_t* splits,
                                         gns_stream_t stream)
{
    using namespace gns;
    if (n <= 0 || w <= 0 || w % (CHUNK / 2) != 0 || keys == nullptr || splits == nullptr) return GNS_ERR_INVALID;
    if (((uintptr_t)keys & 7) || ((uintptr_t)splits & 7)) return GNS_ERR_INVALID;
    const int64_t nblocks = ceil_div(n, CHUNK);
    cudaStream_t s = (cudaStream_t)stream;
    const cudaError_t e = launch(K_MERGE_PARTITION, merge_partition_kernel, dim3((unsigned)ceil_div(nblocks, 256)),
                                 dim3(256), 0, s, keys, n, w, nblocks, splits, (const int*)nullptr);
    return finish_call(e == cudaSuccess ? GNS_OK : GNS_ERR_CUDA, s);
}
