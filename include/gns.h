/*
 * gns.h -- C ABI of the GB300-native stable mergesort after the greeNsort
 * method (J. Oehlschlaegel, "Simple Symmetric Sustainable Sorting -- the
 * greeNsort article", arXiv 2402.01816).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named keys / payload / offsets are DEVICE pointers owned by the
 *   caller (except in gns_sort_host, which takes host pointers).  Sorting is in
 *   place: on return (stream-ordered) keys[0..n) and payload[0..n) hold the
 *   sorted sequence.  keys and payload must not overlap.
 * - Keys are 64-bit (float64 or int64, 8-byte aligned); payloads are uint32
 *   (4-byte aligned).  payload may be NULL (keys only).
 * - Result: the unique stable sort ("Definition of sorting" chapter: the
 *   AscLeft and DescLeft API targets): keys in order from left to right, equal
 *   keys in their input order, for both orders.  DescLeft is not the reverse of
 *   AscLeft: ties keep input order in both.  The key bit patterns are moved,
 *   never canonicalised.
 * - float64 order: IEEE 754 totalOrder: -NaN < -inf < ... < -0.0 < +0.0 < ...
 *   < +inf < +NaN (NaNs by payload bits).  -0.0 and +0.0 are distinct keys.
 * - Calls are asynchronous and ordered on `stream` like CUDA calls.  Errors the
 *   host can see (bad arguments, allocation failure, launch failure) are
 *   returned at once.  Errors found on the device (a bounded wait that ran
 *   out) land in a per-device status word read by gns_stream_status().  With
 *   the environment variable GNS_SYNC_STATUS=1 every call synchronises its
 *   stream and returns that status itself.
 * - Tuning knobs read once per process from the environment (results never
 *   change, only speed): GNS_MERGE_PIPE=ws2|ws3|ws4 (stages of the 100% merge
 *   levels; default ws2), GNS_FROG_PIPE=ws2|ws3|ws4 (the in-place levels;
 *   default ws3), GNS_SEG_SCHEDULE (below).
 * - Workspace: the library allocates only its own scratch, through the
 *   allocator hook (gns_set_allocator; default cudaMallocAsync on `stream`) and
 *   frees it stream-ordered before returning.  gns_workspace_bytes() reports
 *   the size, so %RAM = (12 n + workspace) / 12 n (Sustainability measures
 *   section).
 */
#ifndef GNS_H
#define GNS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL = the legacy default stream. */
typedef struct CUstream_st* gns_stream_t;

/* Return codes (never exceptions). */
enum {
    GNS_OK = 0,
    GNS_ERR_INVALID = -1,      /* bad argument; nothing was launched          */
    GNS_ERR_UNSUPPORTED = -2,  /* valid request this library does not serve  */
    GNS_ERR_OOM = -3,          /* the allocator returned NULL                 */
    GNS_ERR_CUDA = -4,         /* a CUDA runtime call or launch failed        */
    GNS_ERR_TIMEOUT = -5,      /* a device-side bounded wait ran out          */
    GNS_ERR_INTERNAL = -6      /* a device-side consistency check failed      */
};

/* Sort orders: the two stable API targets served (AscLeft, DescLeft). */
enum { GNS_ASCENDING = 0, GNS_DESCENDING = 1 };

/* Key types. */
enum { GNS_KEY_F64 = 0, GNS_KEY_I64 = 1 };

/* Workspace kinds for gns_workspace_bytes. */
enum { GNS_WS_SORT = 0, GNS_WS_LEARNED = 1 };

/*
 * gns_sort -- stable in-place sort of n float64 keys with uint32 payloads.
 *
 * Method: divide & conquer mergesort ("Merging or partitioning?" chapter:
 * split & merge, most work in the merge phases).  Tiles of up to 8192
 * elements are sorted in shared memory; then every merge level is one pass
 * over HBM, split evenly across CTAs by merge-path co-rank search (the
 * "Parallel" section's binary merge over any number of workers).  Before
 * sorting, one read pass detects presorted input (Omitsort / Octosort,
 * "Full adaptivity" section): non-decreasing input is left untouched, strictly
 * decreasing input is reversed once.
 *
 * buffer_fraction selects the memory tier:
 *   >= 1.0      100% distant buffer: Nocopy ping-pong between the keys and an
 *               n-element buffer, the last pass landing in keys ("Forgotten
 *               art": Knuthsort).  Workspace ~ 12 n bytes.
 *   [0.5, 1.0)  <= 50% local buffer: Frogsort1 layout ("Symmetric merging",
 *               "Frogsort1" sections): floor(n/2) buffer slots appended to
 *               the data, left branches data-left, right branches data-right,
 *               merges from the inner ends outward, in place.  Workspace ~ 6 n
 *               bytes.
 *   [1/64, 0.5) Frogsort2 ("Frogsort2" section): the same symmetric merging
 *               with an imbalanced split, inner branch fraction p =
 *               buffer_fraction (rounded to a multiple of 2^-16): a node of m
 *               elements gives floor(p m) to its inner child, and the sort
 *               needs floor(p n) buffer slots (workspace ~ 12 p n bytes).  The
 *               tree is deeper, so the sort does more merge work for less
 *               memory.  The tree is planned on the host and uploaded with a
 *               pageable copy, so this tier cannot be captured in a graph.
 *   < 1/64, NaN GNS_ERR_UNSUPPORTED (< 1/64) / GNS_ERR_INVALID (NaN, negative).
 *
 * Arguments: keys (device, n float64), payload (device, n uint32, or NULL),
 * n >= 0 (n == 0 and n == 1 are no-ops), order GNS_ASCENDING/GNS_DESCENDING.
 * Errors: GNS_ERR_INVALID for n < 0, keys == NULL with n > 0, misaligned
 * pointers, an unknown order; GNS_ERR_OOM; GNS_ERR_CUDA.
 */
int gns_sort(double* keys, uint32_t* payload, int64_t n, int order,
             double buffer_fraction, gns_stream_t stream);

/* gns_sort for int64 keys (two's complement order). */
int gns_sort_i64(int64_t* keys, uint32_t* payload, int64_t n, int order,
                 double buffer_fraction, gns_stream_t stream);

/*
 * gns_sort_symmetric -- the stable sort of gns_sort on an in-place tier's
 * layout (buffer_fraction in [1/64, 1)), in one of the paper's symmetric
 * merging variants:
 *   GNS_FROGSORT1   every node's run stored in the target order (gns_sort's
 *                   in-place tiers; "Frogsort1", "Frogsort2" sections):
 *                   adaptive to presorted input only;
 *   GNS_GECKOSORT1  data-left branches sorted left-ascending and data-right
 *                   branches right-ascending, each merge reading its inner run
 *                   from the far end ("Symmetric merging" section: about 25%
 *                   of the moves saved on ascending and on descending input);
 *   GNS_SQUIDSORT1  the orientation of every run decided by the data
 *                   ("Squidsort" section: Frogsort with Octosort's lazily
 *                   enforced order; Squidsort1 on Frogsort1's tree, Squidsort2
 *                   on Frogsort2's): a leaf tile whose input is non-increasing
 *                   (first key strictly above its last) is stored mirrored, a
 *                   node takes its outer child's orientation, and a mirrored
 *                   root is reversed once at the end, so descending runs --
 *                   ties included -- move only the inner runs' elements per
 *                   level, like ascending ones.
 * buffer_fraction selects the tree as gns_sort does: [0.5, 1) Frogsort1's,
 * [1/64, 0.5) Frogsort2's with inner fraction p = buffer_fraction.  Every
 * variant returns the same bytes as gns_sort (the unique stable sort); they
 * differ only in how much data moves.  Tiles of up to 8192 elements are the
 * leaves.  As gns_sort, one read pass first detects non-decreasing input
 * (nothing to do) and strictly decreasing input (one reversal).
 *
 * Arguments: keys (device, n 64-bit keys of key_type GNS_KEY_F64 or
 * GNS_KEY_I64), payload (device, n uint32, or NULL), n >= 0, order,
 * buffer_fraction, variant.  Workspace as gns_sort at that buffer_fraction.
 * Errors: as gns_sort; GNS_ERR_INVALID for an unknown key type or variant;
 * GNS_ERR_UNSUPPORTED for buffer_fraction >= 1 (no in-place layout) or below
 * 1/64.
 */
enum { GNS_FROGSORT1 = 0, GNS_GECKOSORT1 = 1, GNS_SQUIDSORT1 = 2 };
int gns_sort_symmetric(void* keys, int key_type, uint32_t* payload, int64_t n, int order,
                       double buffer_fraction, int variant, gns_stream_t stream);

/*
 * gns_sort_host -- the same sort on HOST arrays: copies keys and payload to
 * the device on `stream`, sorts them there, copies them back and synchronises
 * the stream.  key_type is GNS_KEY_F64 or GNS_KEY_I64.  Host arrays should be
 * pinned for full copy bandwidth (pageable memory works, slower).  The device
 * copies are workspace (allocator hook).  Errors as gns_sort; the device
 * status word is checked before returning.
 */
int gns_sort_host(void* keys_host, uint32_t* payload_host, int64_t n, int key_type,
                  int order, double buffer_fraction, gns_stream_t stream);

/*
 * gns_segmented_sort -- stable ascending sort of every segment
 * [offsets[s], offsets[s+1]) of an int64 key array independently, in place.
 * No counterpart in the paper (a batching form of the same mergesort): every
 * segment is sorted by the same tile sort and merge passes; segments longer
 * than a tile get only as many merge levels as they need, and each segment's
 * last level lands in keys (the Omitsort idea of the "Full adaptivity" section:
 * the merge decides where the data lies).
 *
 * offsets: device int64[nseg + 1], offsets[0] == 0, non-decreasing (empty
 * segments allowed), offsets[nseg] = total length; not validated on the
 * device.  nseg >= 0.  The whole call is one CUDA-graph launch after its first
 * use for a given (nseg, total length, pointers, stream) -- the graph is
 * captured once and replayed.
 */
int gns_segmented_sort(int64_t* keys, uint32_t* payload, const int64_t* offsets,
                       int64_t nseg, gns_stream_t stream);

/* gns_segmented_sort with a key type and order.  total_n = offsets[nseg] must
 * be passed by the caller (the host never reads device offsets). */
int gns_segmented_sort_ex(void* keys, int key_type, uint32_t* payload,
                          const int64_t* offsets, int64_t nseg, int64_t total_n,
                          int order, gns_stream_t stream);

/*
 * gns_sort_noalloc -- gns_sort at the 100% buffer tier that allocates nothing.
 * (The paper has no counterpart: this is a service for callers, not a step of
 * the method.)
 *
 * Some callers cannot allocate device memory when they need a sort: real-time
 * or signal-safe paths where an allocator call (which may take a lock,
 * synchronise the device or map memory) is not allowed, hosts that reserve all
 * device memory up front and hand a library only the buffers it works on, and
 * code under a fixed memory budget with no room for gns_sort's 12 bytes of
 * scratch per element.  This entry point calls no cudaMalloc, cudaFree,
 * stream-ordered allocator or allocator hook.  Its scratch is one fixed device
 * array inside this library, sized for GNS_NOALLOC_MAX_N elements (about
 * 12 MiB); every GPU that loads the library holds that array until the
 * process exits.  It runs the same passes as gns_sort at buffer_fraction 1.
 *
 * Arguments as gns_sort for float64 keys (device keys, device payload or NULL,
 * n, order); the result is the same stable sort, bit for bit.
 * Errors: GNS_ERR_UNSUPPORTED when n > GNS_NOALLOC_MAX_N (use gns_sort),
 * GNS_ERR_INVALID for bad arguments (as gns_sort, including overlapping keys
 * and payload), GNS_ERR_CUDA if a launch fails.
 *
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture.
 * Sharing: every call on a device uses the same array and the array keeps the
 * last call's contents (the call resets what must start at zero).  Calls that
 * overlap on the GPU -- on different streams, or from different host threads
 * without ordering -- race on the array and corrupt each other's results.
 */
#define GNS_NOALLOC_MAX_N (1 << 20)
int gns_sort_noalloc(double* keys, uint32_t* payload, int64_t n, int order,
                     gns_stream_t stream);

/*
 * Segmented-sort schedule.  The first call for a (total length, segment count,
 * offsets pointer) times the candidate size-class schedules on a scratch copy
 * of the input (synchronising the stream) and keeps the fastest; the call then
 * captures its whole kernel sequence into a CUDA graph, cached with its
 * workspace for these pointers (up to four graphs; the oldest is released).
 * Later calls replay the graph.  Set GNS_SEG_SCHEDULE=0..4 to skip tuning.
 *   gns_segmented_schedule: index of the tuned schedule for this shape
 *     (0 = one 4096-key tile shape for every segment, 1 = segments of up to 1024
 *     keys sorted by 64-thread CTAs, 2 = up to 2048 keys by 128-thread CTAs,
 *     3 and 4 = schedules 0 and 2 with 8192-key tiles by 512-thread CTAs for
 *     the other segments), or -1 if none was tuned yet.
 *   gns_segmented_release: synchronises `stream`, destroys the cached graphs and
 *     frees their workspace, and forgets the tuned schedules.
 */
int gns_segmented_schedule(int64_t total_n, int64_t nseg, const int64_t* offsets);
void gns_segmented_release(gns_stream_t stream);

/*
 * Learned-splitter sort (no counterpart in the paper; a training-system
 * pattern applied to the same stable sort, which it must reproduce exactly).
 *
 * gns_learned_sort sorts float64 keys like gns_sort at the 100% tier, in three
 * phases:
 *   1. fit: 2^16 keys sampled at even strides are sorted.  The CDF model has
 *      two stages: a closed-form first stage, linear interpolation through the
 *      sample quantiles i/64 of the 53-bit prefix of the order-mapped key
 *      (it removes the empty stretches of the key space), and an FP32 MLP
 *      (1 -> 32 tanh -> 32 tanh -> 1 tanh) trained on the device (Adam, mean
 *      squared error) to the residual correction r = 64 (t - x) of that
 *      coordinate x against the sample's empirical CDF t; the estimate is
 *      x + r / 64.
 *   2. partition: the network, evaluated on a 2^16-point grid and made monotone
 *      by a running maximum, proposes 4095 splitters (its inverse at j/4096);
 *      where two splitters coincide (a point mass of the key distribution), the
 *      next one is lowered to one prefix above them, so the mass gets a bucket
 *      of its own.
 *      A key's bucket is the number of splitters at or below its 53-bit prefix
 *      -- an integer, monotone function of the key, so equal keys share a
 *      bucket and the concatenation of stably sorted buckets is exactly the
 *      stable sort, however good or bad the network is.  The 4096-way stable
 *      partition is two 64-way stable scatter passes (low, then high 6 bits of
 *      the bucket).
 *   3. bucket sort: the buckets are ordered, so the array is tile-sorted at
 *      its global 8192-key tiles (a tile may hold the ends of several
 *      buckets) and every bucket that spans tiles is finished by merge levels
 *      over its own runs; buckets whose keys are all bit-identical, which a
 *      stable partition has already left in their final order, are skipped
 *      (the DIET idea of the paper's "DIET-method" section: an all-tied part
 *      needs no sorting); a bucket that came out larger than
 *      `overfull_factor` times the mean is simply sorted by more merge levels
 *      of the same merge path (the plain merge path is the fallback for it).
 *   4. check and fallback: after the bucket sort every bucket is sorted, so its
 *      first and last keys are its minimum and maximum; the check requires the
 *      bucket offsets to partition [0, n) and, at every bucket boundary, the
 *      maximum before it to lie strictly below the minimum after it.  Where
 *      the check fails, the plain
 *      merge sort (gns_sort at the 100% tier) re-sorts the whole array; the
 *      decision is taken on the device (the plain sort's kernels return at
 *      once when the check passes), so the call never waits for the host and
 *      never returns a wrong order, with or without a report.  Equal keys
 *      always share a bucket, so they are still in input order when the plain
 *      sort starts, and its result is the stable sort of the input.
 * buffer_fraction:
 *   >= 1.0      the three phases on the whole array; scratch ~ 16 n bytes for
 *               the partition, then ~ 12 n for the bucket sort (n >= 2^20).
 *   [0.5, 1.0)  half-buffer form (n >= 2^22): the array is the four leaves of
 *               a two-level Frogsort1 tree ("Frogsort1" section: floor(n/2)
 *               buffer slots after the data, here floor(n/2) + 1024).  Leaves
 *               are learned-sorted right to left, each in place with its
 *               scratch carved out of the slots free at that moment, moved to
 *               its gapped data slots, and the tree's two in-place symmetric
 *               merge levels ("Symmetric merging" section) finish the sort.
 *               Scratch ~ 6 n bytes + a few MiB (%RAM about 1.5).
 *   otherwise   (fewer keys, buffer_fraction < 0.5, or no room in the plan)
 *               the whole call is gns_sort at this buffer_fraction, and the
 *               report says fallback = 1.
 * params: NULL = defaults.  report: if not NULL, the call synchronises the
 * stream and fills it (half-buffer form: phase times and bucket counts summed
 * over the four leaves, max_bucket and final_loss their maxima).
 */
typedef struct {
    int train_steps;         /* Adam steps (default 32); 0 = no network:
                                the first stage alone places the splitters
                                (the method without the network)             */
    int batch;               /* samples per step, multiple of 512 (default 1024) */
    float learning_rate;     /* default 1e-2                                  */
    float overfull_factor;   /* bucket counted overfull above this x mean (4) */
} gns_learned_params;

typedef struct {
    int fallback;            /* 1: the call ran gns_sort instead               */
    int nonempty_buckets;
    int64_t max_bucket;      /* largest bucket (keys)                          */
    int overfull_buckets;
    int tied_buckets;        /* buckets whose keys are all equal: left as
                                they are (already the stable order)           */
    float final_loss;        /* training loss of the last step                 */
    float fit_ms, partition_ms, bucket_sort_ms;   /* per-phase device time     */
    int verify_failed;       /* 1: the bucket check failed and the plain
                                merge sort re-sorted the whole array          */
} gns_learned_report;

int gns_learned_sort(double* keys, uint32_t* payload, int64_t n, int order, double buffer_fraction,
                     const gns_learned_params* params, gns_learned_report* report, gns_stream_t stream);

/*
 * The network's own kernels, exposed for gradient checks (device pointers;
 * params packed as [w1(32), b1(32), W2(32x32 row-major: row j holds the
 * inputs of unit j of layer 2), b2(32), w3(32), b3], 1153 floats).
 *   gns_mlp_forward:   y[i] = net(x[i]).
 *   gns_mlp_loss_grad: loss = mean_i (net(x[i]) - t[i])^2 and its gradient
 *                      with respect to the packed params (1153 floats).
 *   gns_mlp_train:     `steps` Adam steps from params_in on (x, t) (m a power
 *                      of two), batch b at step s = samples
 *                      ((s*batch + i) * 40503) mod m, i < batch; writes
 *                      params_out and the last step's loss.
 * Return GNS_OK, GNS_ERR_INVALID or GNS_ERR_CUDA.
 */
int gns_mlp_forward(const float* params, const float* x, int64_t m, float* y, gns_stream_t stream);
int gns_mlp_loss_grad(const float* params, const float* x, const float* t, int64_t m, float* grad,
                      float* loss, gns_stream_t stream);
int gns_mlp_train(const float* x, const float* t, int64_t m, const float* params_in, float* params_out,
                  float* loss_out, int steps, int batch, float learning_rate, gns_stream_t stream);

/* Test hook: plants one fault into the next gns_learned_sort call (consumed
 * by it) to exercise the bucket check and the plain-sort fallback.  The sort
 * must still return the exact stable sort.
 *   GNS_FAULT_BUCKETS_SWAPPED   the partition puts every key of bucket 2k into
 *                               bucket 2k+1 and the other way round (still a
 *                               function of the key, so equal keys stay
 *                               together, but no longer monotone): the bucket
 *                               check fails and the plain merge sort runs;
 *   GNS_FAULT_GARBAGE_WEIGHTS   the network weights are overwritten with NaN
 *                               and +-1e30 before the splitters are derived
 *                               (useless but ordered splitters: overfull
 *                               buckets, sorted by more merge levels);
 *   GNS_FAULT_SPLITTERS_REVERSED the splitter array is reversed before the
 *                               partition.  A key's bucket comes from binary
 *                               searches, whose outcome never decreases with
 *                               the key for any array searched, so the
 *                               partition stays in order and no fallback is
 *                               needed.
 * Any other value clears a pending fault. */
enum { GNS_FAULT_NONE = 0, GNS_FAULT_BUCKETS_SWAPPED = 1, GNS_FAULT_GARBAGE_WEIGHTS = 2,
       GNS_FAULT_SPLITTERS_REVERSED = 3 };
void gns_debug_learned_fault(int kind);

/* Test hook: checks on the host the tree that gns_sort at this buffer_fraction
 * in (0, 1) would run on for n keys (n > 8192): Frogsort1 at [0.5, 1), Frogsort2
 * below ("Symmetric merging", "Frogsort1", "Frogsort2" sections).  Returns 0
 * when every node's children split it exactly (sizes, buffers, adjoining
 * regions and input ranges), every node has at least as many buffer slots as
 * its inner child has elements, the leaves cover the input in order with at
 * most one 8192-key tile each, every data slot lies inside the n + buffer
 * slots, and the chunk numbering is consecutive; else the number (1-6) of the
 * first invariant that fails; -1 for arguments outside that range. */
int gns_frog_plan_check(int64_t n, double buffer_fraction);

/* Test hook: 1 if gns_learned_sort at a buffer_fraction in [0.5, 1) takes its
 * half-buffer form for n keys, with and without a payload (the host-side
 * memory plan fits), else 0.  Runs on the host only. */
int gns_learned_half_plan_ok(int64_t n);

/* The initial network of the learned sort (1153 floats, host memory). */
void gns_mlp_init_params(float* params_host);

/* Size in bytes of the scratch a call allocates.  kind = GNS_WS_SORT for
 * gns_sort at this buffer_fraction, GNS_WS_LEARNED for gns_learned_sort. */
size_t gns_workspace_bytes(int64_t n, double buffer_fraction, int kind);

/*
 * Allocator hook for the library's scratch.  alloc(bytes, stream, ctx) returns
 * device memory usable in stream order on `stream` (or NULL -> GNS_ERR_OOM);
 * free(ptr, stream, ctx) releases it in stream order.  Passing NULL for both
 * restores the default (cudaMallocAsync / cudaFreeAsync).  Process-wide; not
 * to be changed while calls are in flight.
 */
typedef void* (*gns_alloc_fn)(size_t bytes, gns_stream_t stream, void* ctx);
typedef void (*gns_free_fn)(void* ptr, gns_stream_t stream, void* ctx);
void gns_set_allocator(gns_alloc_fn alloc, gns_free_fn free_fn, void* ctx);

/* The default allocator keeps freed workspace in a per-device memory pool for
 * the next call (no unmapping between calls).  This synchronises the current
 * device and returns that cached memory to the driver.  Returns GNS_OK or
 * GNS_ERR_CUDA. */
int gns_release_workspace_cache(void);

/* Synchronises `stream`, returns the current device's status word (GNS_OK or
 * the first device-side error since the last read) and clears it. */
int gns_stream_status(gns_stream_t stream);

/* Static description of a return code. */
const char* gns_strerror(int code);

/* Library version string. */
const char* gns_version(void);

/* --- instrumentation (used by the benchmark; no effect on results) -------- */

/* Number of kernels this library has launched in this process. */
uint64_t gns_launch_count(void);

/* When on (1), every kernel launch is bracketed by CUDA events on its stream;
 * gns_profile_read copies up to `cap` records (kernel id, milliseconds) of the
 * launches since the last read, after synchronising their streams, and returns
 * how many there were.  gns_kernel_name maps an id to its kernel's name. */
void gns_profile_enable(int on);
int gns_profile_read(int* kernel_ids, float* ms, int cap);
const char* gns_kernel_name(int kernel_id);

/* Bounded device waits: the spin limit in nanoseconds (default 2 s) after which
 * a waiting CTA records GNS_ERR_TIMEOUT and returns without writing.  The
 * debug fault `skip_publish_ticket` (>= 0) makes the CTA holding that ticket of
 * the next in-place merge skip publishing its "inputs loaded" flag, so that the
 * wait of the next CTA runs out (used to test the timeout path; -1 = off). */
void gns_set_wait_limit_ns(uint64_t ns);
void gns_debug_skip_publish(int64_t ticket);

/* Test hook (race detection without a sanitizer): every ticket of the in-place
 * merge levels and every leaf of their fused setup waits a pseudo-random time
 * of up to max_ns (at most 50 us; 0 = off, the default) after it is taken and
 * before it loads its inputs.  Tickets then load in perturbed orders, so a
 * store that did not wait for every load it overwrites would change the
 * result; the waits stay far below the wait limit.  Applies to later calls
 * until reset. */
void gns_debug_jitter(uint32_t max_ns);

/* Test hook: the learned sort's bucket sort on its own -- a stable sort of
 * ordered segments.  keys: device, n float64 or int64 keys (key_type) in
 * place; payload: device uint32[n] or NULL; offsets: device int64[nseg + 1],
 * offsets[0] == 0, non-decreasing, offsets[nseg] == n (not validated on the
 * device).  The segments must be ordered under `order`: every key of segment
 * s at or before every key of segment s + 1, equal keys in one segment (the
 * result is undefined otherwise).  The array is tile-sorted at its global
 * 8192-key tiles, each tile sorted whole whatever segment ends it holds, and
 * every segment spanning tiles is finished by merge levels over its own runs;
 * the result is the stable sort of the whole array.  Returns GNS_OK,
 * GNS_ERR_INVALID, GNS_ERR_OOM or GNS_ERR_CUDA. */
int gns_debug_ordered_segments(void* keys, int key_type, uint32_t* payload, int64_t n, const int64_t* offsets,
                               int64_t nseg, int order, gns_stream_t stream);

/* Test hook: the merge-path partition of one Nocopy merge level ("Parallel"
 * section) on its own.  keys: device, n order-mapped 64-bit keys whose
 * consecutive runs of w keys are sorted (w a multiple of 1024); splits:
 * device, ceil(n / 2048) int64.  splits[b] receives the number of elements
 * of the left run among the first b*2048 - p outputs of the stable merge
 * (left run wins ties) of the pair of runs starting at p = floor(b*2048 /
 * 2w) * 2w.  Returns GNS_OK, GNS_ERR_INVALID or GNS_ERR_CUDA. */
int gns_debug_merge_partition(const uint64_t* keys, int64_t n, int64_t w, int64_t* splits,
                              gns_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GNS_H */
