/*
 * gns_oracle.c -- CPU oracle for the stable mergesort hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of the build entry
 * point and the CPU-baseline leg of the benchmark may load this library.  The
 * product path (the CUDA library under paper_2402_01816_gb300/) never calls,
 * links or includes anything from here, and this file includes nothing from
 * there: the two implementations share no code.
 *
 * Everything is plain, sequential, obviously-checkable C:
 *
 *   orc_compare          the total order on 64-bit keys ("Definition of sorting"
 *                        chapter; -0.0/NaN handled by the IEEE 754 totalOrder
 *                        reading).
 *   orc_stable_sort      THE definition of the result: sort (key, input index)
 *                        pairs lexicographically with the C library qsort and
 *                        gather.  Stable sorting has exactly one correct result
 *                        ("Definition of sorting": AscLeft / DescLeft targets).
 *   orc_knuthsort        the paper's prior-art reference mergesort: Nocopy
 *                        alternation between two 100% regions plus Knuth's merge
 *                        with a single exhaustion check ("Forgotten art" section).
 *   orc_frogsort         symmetric merging with at most 50% local buffer:
 *                        Frogsort1 (single-element splits, surplus element to the
 *                        outer side, buffer = N/2 integer division; "Frogsort1"
 *                        section) and Frogsort0 (triplet splits; "Frogsort0"
 *                        section), recursive setup then recursive split & merge,
 *                        merging from the inner to the outer input streams
 *                        ("Symmetric merging" section).
 *   orc_frog_trace       position-label trace of the Frogsort layout after each
 *                        recursion depth, to be compared with the two layout
 *                        tables printed in the Frogsort0 and Frogsort1 sections.
 *   orc_segmented_sort   the definition applied to each segment independently.
 *   orc_final_position   where one input element ends up (rank counting), for
 *                        sampled checks of outputs too large to sort here.
 *
 * Keys are passed as raw 64-bit patterns (float64 or int64); payloads are uint32.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_F64 = 0, ORC_I64 = 1 };
enum { ORC_ASC = 0, ORC_DESC = 1 };

/* ------------------------------------------------------------------------ */
/* Total order                                                                */
/* ------------------------------------------------------------------------ */

/* Ascending total order of two raw key patterns: -1, 0, +1.
 *
 * int64: two's complement signed comparison.
 * float64: IEEE 754 totalOrder.  A key with the sign bit set is below every key
 * without it.  Among non-negative patterns (+0, positive numbers, +inf, +NaN)
 * the unsigned bit patterns order like the magnitudes.  Among negative patterns
 * the order of the magnitudes is reversed.  So -NaN < -inf < ... < -0.0 < +0.0
 * < ... < +inf < +NaN, with NaNs ordered by their payload bits.  The paper does
 * not discuss -0.0 or NaN; this is the reading the library documents. */
int orc_compare(uint64_t a, uint64_t b, int key_type)
{
    if (key_type == ORC_I64) {
        int64_t x = (int64_t)a, y = (int64_t)b;
        return (x < y) ? -1 : (x > y) ? 1 : 0;
    }
    int sa = (int)(a >> 63), sb = (int)(b >> 63);
    if (sa != sb) return sa ? -1 : 1;          /* negative below positive */
    uint64_t ma = a & 0x7fffffffffffffffull, mb = b & 0x7fffffffffffffffull;
    if (ma == mb) return 0;
    if (!sa) return (ma < mb) ? -1 : 1;        /* both non-negative */
    return (ma < mb) ? 1 : -1;                 /* both negative: reversed */
}

/* Order used for a sort call: ascending, or descending (keys non-increasing
 * from left to right).  Ties are never decided here: callers keep input order
 * among equal keys (AscLeft / DescLeft). */
static int ord_cmp(uint64_t a, uint64_t b, int key_type, int order)
{
    int c = orc_compare(a, b, key_type);
    return order == ORC_DESC ? -c : c;
}

/* ------------------------------------------------------------------------ */
/* The definition: sort (key, index) pairs                                    */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t key; int64_t idx; } orc_rec;
static int g_key_type, g_order;   /* qsort has no context argument */

static int rec_cmp(const void* pa, const void* pb)
{
    const orc_rec* a = (const orc_rec*)pa;
    const orc_rec* b = (const orc_rec*)pb;
    int c = ord_cmp(a->key, b->key, g_key_type, g_order);
    if (c) return c;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx) ? 1 : 0;
}

/* Returns 0 on success, -1 on allocation failure. payload may be NULL. */
int orc_stable_sort(uint64_t* keys, uint32_t* payload, int64_t n, int key_type, int order)
{
    if (n <= 1) return 0;
    orc_rec* r = (orc_rec*)malloc((size_t)n * sizeof(orc_rec));
    uint32_t* p = payload ? (uint32_t*)malloc((size_t)n * sizeof(uint32_t)) : NULL;
    if (!r || (payload && !p)) { free(r); free(p); return -1; }
    for (int64_t i = 0; i < n; i++) { r[i].key = keys[i]; r[i].idx = i; }
    if (payload) memcpy(p, payload, (size_t)n * sizeof(uint32_t));
    g_key_type = key_type; g_order = order;
    qsort(r, (size_t)n, sizeof(orc_rec), rec_cmp);
    for (int64_t i = 0; i < n; i++) {
        keys[i] = r[i].key;
        if (payload) payload[i] = p[r[i].idx];
    }
    free(r); free(p);
    return 0;
}

/* Final position of input element i in the stable sort: the number of keys
 * strictly before it in the order, plus the number of equal keys earlier in
 * the input. */
int64_t orc_final_position(const uint64_t* keys, int64_t n, int key_type, int order, int64_t i)
{
    int64_t pos = 0;
    for (int64_t k = 0; k < n; k++) {
        int c = ord_cmp(keys[k], keys[i], key_type, order);
        if (c < 0 || (c == 0 && k < i)) pos++;
    }
    return pos;
}

/* Same as orc_stable_sort, independently per segment [off[s], off[s+1]). */
int orc_segmented_sort(uint64_t* keys, uint32_t* payload, const int64_t* offsets,
                       int64_t nseg, int key_type, int order)
{
    for (int64_t s = 0; s < nseg; s++) {
        int64_t a = offsets[s], len = offsets[s + 1] - offsets[s];
        if (orc_stable_sort(keys + a, payload ? payload + a : NULL, len, key_type, order))
            return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Knuthsort: Nocopy mergesort with Knuth's merge                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    int key_type, order;
    int64_t moves, compares;
} orc_ctx;

/* Merge the sorted runs src[lo..mid) and src[mid..hi) into dst[lo..hi).  Knuth's
 * merge checks for exhaustion only the run whose element was just taken.  Ties
 * take the left run (stability). */
static void knuth_merge(orc_ctx* c, const uint64_t* sk, const uint32_t* sp,
                        uint64_t* dk, uint32_t* dp, int64_t lo, int64_t mid, int64_t hi)
{
    int64_t i = lo, j = mid, k = lo;
    for (;;) {
        c->compares++;
        if (ord_cmp(sk[j], sk[i], c->key_type, c->order) < 0) {
            dk[k] = sk[j]; if (dp) dp[k] = sp[j]; k++; j++; c->moves++;
            if (j == hi) {            /* right run exhausted: copy rest of left */
                while (i < mid) { dk[k] = sk[i]; if (dp) dp[k] = sp[i]; k++; i++; c->moves++; }
                return;
            }
        } else {
            dk[k] = sk[i]; if (dp) dp[k] = sp[i]; k++; i++; c->moves++;
            if (i == mid) {           /* left run exhausted: copy rest of right */
                while (j < hi) { dk[k] = sk[j]; if (dp) dp[k] = sp[j]; k++; j++; c->moves++; }
                return;
            }
        }
    }
}

/* Sort [lo, hi) so that the result lies in (ak, ap), using (bk, bp) which holds
 * an identical copy of the data on entry.  The two halves are sorted into the
 * other region and merged back: the regions alternate per recursion level and
 * no element is ever copied without being merged (Nocopy). */
static void knuth_rec(orc_ctx* c, uint64_t* ak, uint32_t* ap, uint64_t* bk, uint32_t* bp,
                      int64_t lo, int64_t hi)
{
    if (hi - lo < 2) return;
    int64_t mid = lo + (hi - lo) / 2;
    knuth_rec(c, bk, bp, ak, ap, lo, mid);
    knuth_rec(c, bk, bp, ak, ap, mid, hi);
    knuth_merge(c, bk, bp, ak, ap, lo, mid, hi);
}

/* counters (may be NULL): [0] = element moves (including the initial copy into
 * the buffer), [1] = key comparisons.  Returns 0, or -1 on allocation failure. */
int orc_knuthsort(uint64_t* keys, uint32_t* payload, int64_t n, int key_type, int order,
                  int64_t* counters)
{
    orc_ctx c = { key_type, order, 0, 0 };
    if (n >= 2) {
        uint64_t* bk = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
        uint32_t* bp = payload ? (uint32_t*)malloc((size_t)n * sizeof(uint32_t)) : NULL;
        if (!bk || (payload && !bp)) { free(bk); free(bp); return -1; }
        memcpy(bk, keys, (size_t)n * sizeof(uint64_t));
        if (payload) memcpy(bp, payload, (size_t)n * sizeof(uint32_t));
        c.moves += n;
        knuth_rec(&c, keys, payload, bk, bp, 0, n);
        free(bk); free(bp);
    }
    if (counters) { counters[0] = c.moves; counters[1] = c.compares; }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Frogsort: symmetric merging with <= 50% local buffer                       */
/* ------------------------------------------------------------------------ */
/*
 * A node sorts n elements inside a region of n + b slots.  A "data-left" node
 * ends with its data in the left n slots and its buffer on the right (Ab); a
 * "data-right" node ends with buffer left, data right (aB).  The left child of
 * every node is data-left and the right child data-right, so the two children's
 * buffers meet in the middle of the parent's region.  The parent then merges
 * from the inner ends of the two runs outward, and the result is aligned at the
 * parent's outer border:
 *   data-left parent : write from slot n-1 down to 0, larger key first; on ties
 *                      the right run's element is written (it is later in the
 *                      input, so it belongs at the higher slot).
 *   data-right parent: write from slot b up to n+b-1, smaller key first; on ties
 *                      the left run's element is written.
 * The outer side of a data-left node is its left, of a data-right node its
 * right.  Split rule: an odd surplus element goes to the outer child.  Buffer
 * rule: the root has b = floor(n/2); the outer child gets floor(n_outer/2) and
 * the inner child the rest of the parent's buffer.  (The paper gives only the
 * root's buffer; this split reproduces both of its layout tables and gives
 * every node at least as much buffer as its inner child has elements, which is
 * what the in-place merge needs.)
 *
 * split_unit g: 1 = Frogsort1 (single-element splits); 2 = Frogsort0 (the
 * triplet variant: a node of k triplets holds n = 2k elements and splits into
 * ceil(k/2) outer and floor(k/2) inner triplets; a single triplet splits into
 * its two elements).
 */

typedef struct {
    int64_t n, b;       /* elements, buffer slots */
    int64_t r;          /* first slot of the region */
    int64_t s;          /* first input index of the node's elements */
    int side;           /* 0 = data-left, 1 = data-right */
    int depth;
} frog_node;

static void frog_children(const frog_node* p, int g, frog_node* L, frog_node* R)
{
    int64_t n_outer;
    if (g == 2 && p->n >= 4 && p->n % 2 == 0) {
        int64_t k = p->n / 2;
        n_outer = 2 * ((k + 1) / 2);
    } else {
        n_outer = (p->n + 1) / 2;
    }
    int64_t n_inner = p->n - n_outer;
    int64_t b_outer = n_outer / 2;
    int64_t b_inner = p->b - b_outer;
    L->side = 0; R->side = 1;
    L->depth = R->depth = p->depth + 1;
    if (p->side == 0) { L->n = n_outer; L->b = b_outer; R->n = n_inner; R->b = b_inner; }
    else              { L->n = n_inner; L->b = b_inner; R->n = n_outer; R->b = b_outer; }
    L->r = p->r;            R->r = p->r + L->n + L->b;
    L->s = p->s;            R->s = p->s + L->n;
}

/* First slot of a node's data in its final layout. */
static int64_t frog_data_slot(const frog_node* x)
{
    return x->side == 0 ? x->r : x->r + x->b;
}

/* Setup recursion: destination slot of every input element (its leaf's slot). */
static void frog_setup_dest(const frog_node* x, int g, int64_t* dest)
{
    if (x->n == 1) { dest[x->s] = frog_data_slot(x); return; }
    frog_node L, R;
    frog_children(x, g, &L, &R);
    frog_setup_dest(&L, g, dest);
    frog_setup_dest(&R, g, dest);
}

typedef struct {
    orc_ctx c;
    int g;
    int stop_depth;      /* merge only nodes with depth >= stop_depth */
    uint64_t* k;         /* n + b slots */
    uint32_t* p;         /* n + b slots or NULL */
    int32_t* label;      /* optional: slot labels for the layout trace */
} frog_run;

static void frog_move(frog_run* f, int64_t to, int64_t from)
{
    f->k[to] = f->k[from];
    if (f->p) f->p[to] = f->p[from];
    if (f->label) f->label[to] = f->label[from];
    f->c.moves++;
}

/* After a node's merge, the labels of its buffer slots are re-assigned: the
 * buffer labels that were in the region are handed out to the free slots in
 * increasing order (this is how the paper's tables print the buffer). */
static void frog_relabel_buffer(frog_run* f, const frog_node* x, const int32_t* before)
{
    if (!f->label || x->b == 0) return;
    int64_t nb = 0, m = x->n + x->b;
    int32_t* bl = (int32_t*)malloc((size_t)x->b * sizeof(int32_t));
    for (int64_t i = 0; i < m; i++)
        if (before[i] < 0) bl[nb++] = before[i];
    /* buffer labels are stored negative: -(position+1); increasing position
     * order is decreasing stored value */
    for (int64_t a = 0; a < nb; a++)
        for (int64_t z = a + 1; z < nb; z++)
            if (bl[z] > bl[a]) { int32_t t = bl[a]; bl[a] = bl[z]; bl[z] = t; }
    int64_t b0 = x->side == 0 ? x->r + x->n : x->r;
    for (int64_t i = 0; i < nb; i++) f->label[b0 + i] = bl[i];
    free(bl);
}

static void frog_merge(frog_run* f, const frog_node* x, const frog_node* L, const frog_node* R)
{
    int kt = f->c.key_type, od = f->c.order;
    int64_t m = x->n + x->b;
    int32_t* before = NULL;
    if (f->label) {
        before = (int32_t*)malloc((size_t)m * sizeof(int32_t));
        memcpy(before, f->label + x->r, (size_t)m * sizeof(int32_t));
    }
    int64_t la = frog_data_slot(L), lz = la + L->n;   /* left run  [la, lz) */
    int64_t ra = frog_data_slot(R), rz = ra + R->n;   /* right run [ra, rz) */
    if (x->side == 0) {
        /* write downward from the inner end of the output [r, r+n) */
        int64_t i = lz - 1, j = rz - 1, w = x->r + x->n - 1;
        while (j >= ra) {
            if (i < la) { frog_move(f, w--, j--); continue; }
            f->c.compares++;
            if (ord_cmp(f->k[j], f->k[i], kt, od) >= 0) frog_move(f, w--, j--);
            else frog_move(f, w--, i--);
        }
        /* right run exhausted: the rest of the left run is already in place */
    } else {
        /* write upward from the inner end of the output [r+b, r+n+b) */
        int64_t i = la, j = ra, w = x->r + x->b;
        while (i < lz) {
            if (j >= rz) { frog_move(f, w++, i++); continue; }
            f->c.compares++;
            if (ord_cmp(f->k[i], f->k[j], kt, od) <= 0) frog_move(f, w++, i++);
            else frog_move(f, w++, j++);
        }
        /* left run exhausted: the rest of the right run is already in place */
    }
    if (f->label) {
        /* mark every non-data slot of the region as buffer again */
        int64_t d0 = frog_data_slot(x);
        for (int64_t q = x->r; q < x->r + m; q++)
            if (q < d0 || q >= d0 + x->n) f->label[q] = 0;
        frog_relabel_buffer(f, x, before);
        free(before);
    }
}

static void frog_sort_rec(frog_run* f, const frog_node* x)
{
    if (x->n == 1) return;
    frog_node L, R;
    frog_children(x, f->g, &L, &R);
    frog_sort_rec(f, &L);
    frog_sort_rec(f, &R);
    if (x->depth >= f->stop_depth) frog_merge(f, x, &L, &R);
}

static frog_node frog_root(int64_t n, int g)
{
    frog_node root;
    root.n = n; root.b = n / 2; root.r = 0; root.s = 0; root.side = 0; root.depth = 0;
    (void)g;
    return root;
}

/* Buffer slots Frogsort needs for n elements (the paper's N/2). */
int64_t orc_frog_buffer(int64_t n) { return n / 2; }

/* Sort in place using n/2 extra slots.  counters (may be NULL): [0] setup moves,
 * [1] merge moves, [2] merge comparisons.  split_unit 2 requires even n. */
int orc_frogsort(uint64_t* keys, uint32_t* payload, int64_t n, int key_type, int order,
                 int split_unit, int64_t* counters)
{
    if (split_unit == 2 && (n % 2)) return -2;
    int64_t setup_moves = 0;
    frog_run f;
    memset(&f, 0, sizeof(f));
    f.c.key_type = key_type; f.c.order = order; f.g = split_unit; f.stop_depth = 0;
    if (n >= 2) {
        int64_t b = n / 2, m = n + b;
        f.k = (uint64_t*)malloc((size_t)m * sizeof(uint64_t));
        f.p = payload ? (uint32_t*)malloc((size_t)m * sizeof(uint32_t)) : NULL;
        int64_t* dest = (int64_t*)malloc((size_t)n * sizeof(int64_t));
        if (!f.k || (payload && !f.p) || !dest) { free(f.k); free(f.p); free(dest); return -1; }
        /* the caller's n slots followed by the buffer's b slots */
        memcpy(f.k, keys, (size_t)n * sizeof(uint64_t));
        if (payload) memcpy(f.p, payload, (size_t)n * sizeof(uint32_t));
        frog_node root = frog_root(n, split_unit);
        frog_setup_dest(&root, split_unit, dest);
        /* every element moves right (dest >= source) and dest increases with the
         * source index, so moving from the highest element down never
         * overwrites an element that has not moved yet */
        for (int64_t e = n - 1; e >= 0; e--) {
            if (dest[e] != e) {
                f.k[dest[e]] = f.k[e];
                if (payload) f.p[dest[e]] = f.p[e];
                setup_moves++;
            }
        }
        free(dest);
        frog_sort_rec(&f, &root);
        memcpy(keys, f.k, (size_t)n * sizeof(uint64_t));
        if (payload) memcpy(payload, f.p, (size_t)n * sizeof(uint32_t));
        free(f.k); free(f.p);
    }
    if (counters) { counters[0] = setup_moves; counters[1] = f.c.moves; counters[2] = f.c.compares; }
    return 0;
}

/* ------------------------------------------------------------------------
 * Frogsort2 (Frogsort2 section): symmetric merging with an imbalanced split.
 * With inner fraction p (here p_num / p_den <= 1/2) the inner branch of a
 * node of n elements holds floor(p n) of them, and the whole sort needs only
 * floor(p n) buffer slots.  Reading (the section gives only "inner branch
 * p%, p% buffer"):
 *   root:   n elements, b = floor(p n) buffer slots;
 *   split:  n_inner = floor(p n), n_outer = n - n_inner;
 *           b_outer = floor(p n_outer), b_inner = b - b_outer;
 *   leaves: nodes of at most `leaf` elements, stably sorted into their data
 *           slots at setup (the base case), every other node merged as in
 *           Frogsort1 (frog_merge above: inner end to outer end).
 * By induction every node keeps b >= floor(p n) = n_inner (floor(x) -
 * floor(y) >= floor(x - y)), which is what the in-place merge needs; the code
 * checks it anyway.  With p = 1/2 and leaf = 1 the split is Frogsort1's.
 * ------------------------------------------------------------------------ */
typedef struct {
    int64_t pn, pd;     /* p = pn / pd */
    int64_t leaf;
    int bad;            /* set if a node breaks b >= n_inner */
} frog2_cfg;

static int64_t frog2_floor_p(const frog2_cfg* c, int64_t n) { return (n * c->pn) / c->pd; }

static void frog2_children(const frog2_cfg* c, const frog_node* p, frog_node* L, frog_node* R)
{
    int64_t n_inner = frog2_floor_p(c, p->n), n_outer = p->n - n_inner;
    int64_t b_outer = frog2_floor_p(c, n_outer), b_inner = p->b - b_outer;
    L->side = 0; R->side = 1;
    L->depth = R->depth = p->depth + 1;
    if (p->side == 0) { L->n = n_outer; L->b = b_outer; R->n = n_inner; R->b = b_inner; }
    else              { L->n = n_inner; L->b = b_inner; R->n = n_outer; R->b = b_outer; }
    L->r = p->r;            R->r = p->r + L->n + L->b;
    L->s = p->s;            R->s = p->s + L->n;
}

static int frog2_is_leaf(const frog2_cfg* c, const frog_node* x)
{
    return x->n <= c->leaf || frog2_floor_p(c, x->n) == 0;
}

static void frog2_setup_dest(frog2_cfg* c, const frog_node* x, int64_t* dest)
{
    if (frog2_is_leaf(c, x)) {
        for (int64_t e = 0; e < x->n; e++) dest[x->s + e] = frog_data_slot(x) + e;
        return;
    }
    frog_node L, R;
    frog2_children(c, x, &L, &R);
    frog2_setup_dest(c, &L, dest);
    frog2_setup_dest(c, &R, dest);
}

/* the base case: a stable insertion sort of a leaf's slots */
static void frog2_sort_leaf(frog_run* f, const frog_node* x)
{
    int64_t a = frog_data_slot(x), z = a + x->n;
    for (int64_t i = a + 1; i < z; i++) {
        uint64_t k = f->k[i];
        uint32_t v = f->p ? f->p[i] : 0;
        int64_t j = i - 1;
        while (j >= a) {
            f->c.compares++;
            if (ord_cmp(f->k[j], k, f->c.key_type, f->c.order) <= 0) break;
            f->k[j + 1] = f->k[j];
            if (f->p) f->p[j + 1] = f->p[j];
            j--;
        }
        f->k[j + 1] = k;
        if (f->p) f->p[j + 1] = v;
    }
}

static void frog2_sort_rec(frog2_cfg* c, frog_run* f, const frog_node* x)
{
    if (frog2_is_leaf(c, x)) {
        frog2_sort_leaf(f, x);
        return;
    }
    frog_node L, R;
    frog2_children(c, x, &L, &R);
    if (x->b < (x->side == 0 ? R.n : L.n)) c->bad = 1;   /* the inner child must fit the buffer */
    frog2_sort_rec(c, f, &L);
    frog2_sort_rec(c, f, &R);
    frog_merge(f, x, &L, &R);
}

/* Buffer slots Frogsort2 needs for n elements: floor(p n). */
int64_t orc_frog2_buffer(int64_t n, int64_t p_num, int64_t p_den) { return (n * p_num) / p_den; }

/* Sort in place using floor(p n) extra slots, p = p_num / p_den in (0, 1/2];
 * leaf >= 1.  counters as orc_frogsort.  Returns 0, -1 (allocation), -2
 * (bad arguments) or -3 (a node broke b >= n_inner: cannot happen). */
int orc_frogsort2(uint64_t* keys, uint32_t* payload, int64_t n, int key_type, int order, int64_t p_num,
                  int64_t p_den, int64_t leaf, int64_t* counters)
{
    if (p_num <= 0 || p_den <= 0 || 2 * p_num > p_den || leaf < 1) return -2;
    frog2_cfg c = {p_num, p_den, leaf, 0};
    int64_t setup_moves = 0;
    frog_run f;
    memset(&f, 0, sizeof(f));
    f.c.key_type = key_type; f.c.order = order;
    if (n >= 2) {
        int64_t b = frog2_floor_p(&c, n), m = n + b;
        f.k = (uint64_t*)malloc((size_t)m * sizeof(uint64_t));
        f.p = payload ? (uint32_t*)malloc((size_t)m * sizeof(uint32_t)) : NULL;
        int64_t* dest = (int64_t*)malloc((size_t)n * sizeof(int64_t));
        if (!f.k || (payload && !f.p) || !dest) { free(f.k); free(f.p); free(dest); return -1; }
        memcpy(f.k, keys, (size_t)n * sizeof(uint64_t));
        if (payload) memcpy(f.p, payload, (size_t)n * sizeof(uint32_t));
        frog_node root;
        root.n = n; root.b = b; root.r = 0; root.s = 0; root.side = 0; root.depth = 0;
        frog2_setup_dest(&c, &root, dest);
        for (int64_t e = n - 1; e >= 0; e--) {      /* dest >= source, increasing: top down */
            if (dest[e] != e) {
                f.k[dest[e]] = f.k[e];
                if (payload) f.p[dest[e]] = f.p[e];
                setup_moves++;
            }
        }
        free(dest);
        frog2_sort_rec(&c, &f, &root);
        memcpy(keys, f.k, (size_t)n * sizeof(uint64_t));
        if (payload) memcpy(payload, f.p, (size_t)n * sizeof(uint32_t));
        free(f.k); free(f.p);
    }
    if (counters) { counters[0] = setup_moves; counters[1] = f.c.moves; counters[2] = f.c.compares; }
    return c.bad ? -3 : 0;
}

/* Depth of the Frogsort tree for n elements (leaves are single elements). */
static int frog_depth_rec(const frog_node* x, int g)
{
    if (x->n == 1) return x->depth;
    frog_node L, R;
    frog_children(x, g, &L, &R);
    int a = frog_depth_rec(&L, g), z = frog_depth_rec(&R, g);
    return a > z ? a : z;
}

int orc_frog_depth(int64_t n, int split_unit)
{
    frog_node root = frog_root(n, split_unit);
    return n >= 1 ? frog_depth_rec(&root, split_unit) : 0;
}

/* Layout trace on presorted keys (key = setup slot), recording slot labels.
 * labels_out has (D+1) rows of n + n/2 entries, D = depth of the deepest leaf:
 * row 0 = after setup, row t = after the merges of every node at depth >= D - t
 * (t merge levels, bottom-up).  A label is +(slot+1) for the data element
 * that was set up in that slot, -(slot+1) for the buffer slot labelled by its
 * setup slot.  Returns the number of rows, or -1. */
int orc_frog_trace(int64_t n, int split_unit, int32_t* labels_out, int max_rows)
{
    if (n < 1 || (split_unit == 2 && (n % 2))) return -1;
    int D = orc_frog_depth(n, split_unit);
    if (D + 1 > max_rows) return -1;
    int64_t b = n / 2, m = n + b;
    frog_node root = frog_root(n, split_unit);
    int64_t* dest = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    frog_setup_dest(&root, split_unit, dest);
    for (int row = 0; row <= D; row++) {
        frog_run f;
        memset(&f, 0, sizeof(f));
        f.c.key_type = ORC_I64; f.c.order = ORC_ASC; f.g = split_unit;
        f.stop_depth = D - row;   /* row t: merges at depths >= D - t */
        f.k = (uint64_t*)calloc((size_t)m, sizeof(uint64_t));
        f.label = (int32_t*)malloc((size_t)m * sizeof(int32_t));
        char* is_data = (char*)calloc((size_t)m, 1);
        for (int64_t e = 0; e < n; e++) is_data[dest[e]] = 1;
        for (int64_t q = 0; q < m; q++) {
            f.label[q] = is_data[q] ? (int32_t)(q + 1) : -(int32_t)(q + 1);
            f.k[q] = (uint64_t)q;   /* presorted by setup slot */
        }
        if (row > 0) frog_sort_rec(&f, &root);
        memcpy(labels_out + (size_t)row * (size_t)m, f.label, (size_t)m * sizeof(int32_t));
        free(f.k); free(f.label); free(is_data);
    }
    free(dest);
    return D + 1;
}

/* ========================================================================
 * Orientations ("Definition of sorting" chapter: the four stable API
 * targets).  The adaptive sorts below let a node return its sorted data in
 * either of two orientations: ORI_ASC is the target itself (AscLeft: keys in
 * order from left to right, ties in input order); ORI_DESC is its mirror image
 * (AscRight: the same sequence stored right to left).  A single element is
 * both (ORI_ANY).  Element e (0-based, in AscLeft order) of a run of n stored
 * at slot a in orientation o sits at slot a + e (ORI_ASC) or a + n - 1 - e
 * (ORI_DESC).
 * ======================================================================== */
enum { ORI_ASC = 0, ORI_DESC = 1, ORI_ANY = 2 };

static int64_t ori_slot(int ori, int64_t a, int64_t n, int64_t e)
{
    return ori == ORI_DESC ? a + n - 1 - e : a + e;
}

/* ------------------------------------------------------------------------
 * Omitsort and Octosort ("Full adaptivity" section), 100% buffer.
 *
 * Omitsort: top-down mergesort (Knuthsort's split, left = floor(n/2)) over two
 * regions, the caller's array (region 0) and an n-slot buffer (region 1).
 * Instead of Nocopy's fixed alternation, every sort returns the region its
 * data ended in.  If the two halves ended in different regions, the half in
 * the buffer is copied to the data region first.  Then one comparison of the
 * two elements at the halves' boundary decides whether they overlap; if not,
 * the merge is omitted and the node stays where it is, else the halves are
 * merged into the other region.  At the end the data is copied back if it
 * lies in the buffer.  Presorted input costs n - 1 comparisons and no move.
 *
 * Octosort: Omitsort whose nodes return an orientation as well, decided by the
 * data.  Two single elements take ORI_DESC when they are strictly out of
 * order, else ORI_ASC (one comparison, no move).  Children of the same
 * orientation (a single element adopts its sibling's) are tested for overlap
 * in that orientation (ORI_ASC: left's last <= right's first; ORI_DESC: the
 * left's last element strictly above the right's first, because the mirror
 * image keeps the later of two equal keys on the left) and merged in it when
 * they overlap.  Only when the children disagree is the desired order
 * enforced: they are merged into ORI_ASC, the ORI_DESC child read from its
 * far end.  A root in ORI_DESC is reversed once at the end, so strictly
 * descending input costs n - 1 comparisons and one reversal.
 * ------------------------------------------------------------------------ */
typedef struct {
    orc_ctx c;
    int lazy;               /* 0 = Omitsort, 1 = Octosort */
    uint64_t* k[2];
    uint32_t* p[2];         /* NULL when there is no payload */
} omit_run;

typedef struct { int reg, ori; } omit_res;

static void om_put(omit_run* f, int dr, int64_t d, int sr, int64_t s)
{
    f->k[dr][d] = f->k[sr][s];
    if (f->p[0]) f->p[dr][d] = f->p[sr][s];
    f->c.moves++;
}

/* Out-of-place merge of the runs [lo, lo+nl) (orientation oL) and
 * [lo+nl, lo+n) (orientation oR) of region r into region 1-r, stored in
 * orientation o.  Both runs are walked in AscLeft order; ties take the left
 * run (stability); Knuth's single exhaustion check per step. */
static void om_merge(omit_run* f, int r, int64_t lo, int64_t nl, int oL, int64_t nr, int oR, int o)
{
    const int kt = f->c.key_type, od = f->c.order;
    const int64_t n = nl + nr;
    int64_t i = 0, j = 0, t = 0;
    const uint64_t* sk = f->k[r];
    for (;;) {
        int64_t a = ori_slot(oL, lo, nl, i), b = ori_slot(oR, lo + nl, nr, j);
        f->c.compares++;
        if (ord_cmp(sk[b], sk[a], kt, od) < 0) {
            om_put(f, 1 - r, ori_slot(o, lo, n, t++), r, b);
            if (++j == nr) {
                for (; i < nl; i++) om_put(f, 1 - r, ori_slot(o, lo, n, t++), r, ori_slot(oL, lo, nl, i));
                return;
            }
        } else {
            om_put(f, 1 - r, ori_slot(o, lo, n, t++), r, a);
            if (++i == nl) {
                for (; j < nr; j++) om_put(f, 1 - r, ori_slot(o, lo, n, t++), r, ori_slot(oR, lo + nl, nr, j));
                return;
            }
        }
    }
}

static omit_res om_rec(omit_run* f, int64_t lo, int64_t n)
{
    omit_res res = {0, f->lazy ? ORI_ANY : ORI_ASC};
    if (n == 1) return res;
    const int64_t nl = n / 2, nr = n - nl, m = lo + nl;
    omit_res a = om_rec(f, lo, nl), b = om_rec(f, m, nr);
    if (a.reg != b.reg) {                 /* bring the half in the buffer to the data region */
        if (a.reg == 1) for (int64_t e = lo; e < m; e++) om_put(f, 0, e, 1, e);
        else            for (int64_t e = m; e < lo + n; e++) om_put(f, 0, e, 1, e);
        a.reg = b.reg = 0;
    }
    const int r = a.reg, kt = f->c.key_type, od = f->c.order;
    const uint64_t* k = f->k[r];
    res.reg = r;
    if (a.ori == ORI_ANY && b.ori == ORI_ANY) {       /* Octosort: two single elements */
        f->c.compares++;
        res.ori = ord_cmp(k[m], k[m - 1], kt, od) < 0 ? ORI_DESC : ORI_ASC;
        return res;                                   /* in either orientation already */
    }
    const int oL = a.ori == ORI_ANY ? b.ori : a.ori;
    const int oR = b.ori == ORI_ANY ? a.ori : b.ori;
    if (oL != oR) {                                   /* disagreement: enforce the target */
        om_merge(f, r, lo, nl, oL, nr, oR, ORI_ASC);
        res.reg = 1 - r;
        res.ori = ORI_ASC;
        return res;
    }
    f->c.compares++;                                  /* the non-overlap test */
    const int c = ord_cmp(k[m - 1], k[m], kt, od);
    if (oL == ORI_ASC ? c <= 0 : c > 0) {
        res.ori = oL;                                 /* omitted: no move */
        return res;
    }
    om_merge(f, r, lo, nl, oL, nr, oR, oL);
    res.reg = 1 - r;
    res.ori = oL;
    return res;
}

/* lazy = 0: Omitsort, 1: Octosort.  counters (may be NULL): [0] element moves
 * (merges, region fix-up copies, the final copy or reversal), [1] comparisons.
 * Returns 0, or -1 on allocation failure. */
int orc_omitsort(uint64_t* keys, uint32_t* payload, int64_t n, int key_type, int order, int lazy,
                 int64_t* counters)
{
    omit_run f;
    memset(&f, 0, sizeof(f));
    f.c.key_type = key_type; f.c.order = order; f.lazy = lazy ? 1 : 0;
    if (n >= 2) {
        f.k[0] = keys; f.p[0] = payload;
        f.k[1] = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
        f.p[1] = payload ? (uint32_t*)malloc((size_t)n * sizeof(uint32_t)) : NULL;
        if (!f.k[1] || (payload && !f.p[1])) { free(f.k[1]); free(f.p[1]); return -1; }
        omit_res res = om_rec(&f, 0, n);
        if (res.ori == ORI_DESC) {                    /* the one final reversal */
            if (res.reg == 1) {
                for (int64_t e = 0; e < n; e++) om_put(&f, 0, e, 1, n - 1 - e);
            } else {
                for (int64_t i = 0, j = n - 1; i < j; i++, j--) {
                    uint64_t tk = keys[i]; keys[i] = keys[j]; keys[j] = tk;
                    if (payload) { uint32_t tp = payload[i]; payload[i] = payload[j]; payload[j] = tp; }
                    f.c.moves += 2;
                }
            }
        } else if (res.reg == 1) {
            for (int64_t e = 0; e < n; e++) om_put(&f, 0, e, 1, e);
        }
        free(f.k[1]); free(f.p[1]);
    }
    if (counters) { counters[0] = f.c.moves; counters[1] = f.c.compares; }
    return 0;
}

/* ------------------------------------------------------------------------
 * Geckosort1 and Squidsort1: symmetric merging ("Symmetric merging" and
 * "Squidsort" sections) on Frogsort1's tree, buffer and setup (frog_children,
 * frog_setup_dest above), with nodes in either orientation.
 *
 * The in-place merge of a node (sym_merge) writes from the inner end of the
 * node's output outward (data-left node: from slot r+n-1 down; data-right
 * node: from slot r+b up) and reads each run from the end whose element is
 * written first.  The outer child's run lies under the output, so it must be
 * read from its inner end, which fixes the node's orientation to the outer
 * child's; the inner child lies in the buffer, beyond the output, and can be
 * read from either end, so its orientation is free.  With the orientation o
 * of the node, the element written first is the largest and latest
 * ("largest first") when a data-left node is ORI_ASC or a data-right node
 * ORI_DESC, else the smallest and earliest ("smallest first").  Largest first
 * takes the right run on ties (its elements are later in the input), smallest
 * first takes the left run.  The merge stops when the inner child is used
 * up: the rest of the outer child is then in its final slots.
 *
 * Geckosort1: every data-left node is ORI_ASC and every data-right node
 * ORI_DESC (one branch sorted left-ascending, the other right-ascending, the
 * right branch the mirror image of the left).  On ascending input a data-left
 * node moves only its inner child and a data-right node moves everything; on
 * descending input the other way round: 25% fewer moves for either order.
 *
 * Squidsort1: the orientation is decided by the data (Octosort's lazily
 * enforced order): two single elements take ORI_DESC when they are strictly
 * out of order (one comparison, which is also their non-overlap test); any
 * larger node takes its outer child's orientation (the one the in-place merge
 * can produce; a single element adopts its sibling's).  Every larger node
 * first compares the inner child's last element in write order with the outer
 * child's first (the non-overlap test); when the inner child comes entirely
 * first it is moved next to the outer child without further comparisons.
 * A root in ORI_DESC is reversed once at the end.  Presorted and strictly
 * descending inputs cost one comparison per node and move half the elements
 * per level (plus the one reversal for the latter).
 * ------------------------------------------------------------------------ */
typedef struct {
    frog_run f;
    int lazy;           /* 0 = Geckosort1, 1 = Squidsort1 */
} sym_run;

/* Slot of the t-th element of child x (orientation o) in write order. */
static int64_t sym_slot(const frog_node* x, int o, int largest_first, int64_t t)
{
    const int64_t e = largest_first ? x->n - 1 - t : t;    /* position in AscLeft order */
    return ori_slot(o, frog_data_slot(x), x->n, e);
}

static void sym_merge(sym_run* s, const frog_node* x, const frog_node* L, int oL, const frog_node* R, int oR,
                      int o, int test_overlap)
{
    frog_run* f = &s->f;
    const int kt = f->c.key_type, od = f->c.order;
    const int lf = (x->side == 0) == (o == ORI_ASC);
    int64_t w = x->side == 0 ? x->r + x->n - 1 : x->r + x->b;
    const int64_t step = x->side == 0 ? -1 : 1;
    const frog_node* I = x->side == 0 ? R : L;         /* inner child */
    const frog_node* O = x->side == 0 ? L : R;         /* outer child */
    const int oI = x->side == 0 ? oR : oL, oO = x->side == 0 ? oL : oR;
    int64_t i = 0, j = 0;                               /* taken from L, from R */
    /* element a of L goes before element b of R in write order */
#define SYM_L_FIRST(a, b) (lf ? ord_cmp(f->k[a], f->k[b], kt, od) > 0 : ord_cmp(f->k[a], f->k[b], kt, od) <= 0)
    if (test_overlap) {
        const int64_t il = sym_slot(I, oI, lf, I->n - 1), of = sym_slot(O, oO, lf, 0);
        f->c.compares++;
        const int inner_first = x->side == 0 ? !SYM_L_FIRST(of, il) : SYM_L_FIRST(il, of);
        if (inner_first) {
            for (int64_t t = 0; t < I->n; t++, w += step) frog_move(f, w, sym_slot(I, oI, lf, t));
            return;
        }
    }
    while (x->side == 0 ? j < R->n : i < L->n) {
        int take_l;
        if (i == L->n) take_l = 0;
        else if (j == R->n) take_l = 1;
        else {
            f->c.compares++;
            take_l = SYM_L_FIRST(sym_slot(L, oL, lf, i), sym_slot(R, oR, lf, j));
        }
        if (take_l) frog_move(f, w, sym_slot(L, oL, lf, i++));
        else        frog_move(f, w, sym_slot(R, oR, lf, j++));
        w += step;
    }
#undef SYM_L_FIRST
}

static int sym_rec(sym_run* s, const frog_node* x)
{
    if (x->n == 1) return ORI_ANY;
    frog_node L, R;
    frog_children(x, 1, &L, &R);
    int oL = sym_rec(s, &L), oR = sym_rec(s, &R);
    if (!s->lazy) {                                     /* Geckosort1: orientation by side */
        if (oL == ORI_ANY) oL = ORI_ASC;
        if (oR == ORI_ANY) oR = ORI_DESC;
        const int o = x->side == 0 ? ORI_ASC : ORI_DESC;
        sym_merge(s, x, &L, oL, &R, oR, o, 0);
        return o;
    }
    if (oL == ORI_ANY && oR == ORI_ANY) {               /* Squidsort1: the data decides */
        const frog_run* f = &s->f;
        s->f.c.compares++;
        const int o = ord_cmp(f->k[frog_data_slot(&R)], f->k[frog_data_slot(&L)], f->c.key_type, f->c.order) < 0
                          ? ORI_DESC : ORI_ASC;
        /* the comparison also settles the order: the inner element is moved next to the outer one */
        const frog_node* I = x->side == 0 ? &R : &L;
        const int64_t w = x->side == 0 ? x->r + x->n - 1 : x->r + x->b;
        frog_move(&s->f, w, frog_data_slot(I));
        return o;
    }
    if (oL == ORI_ANY) oL = oR;
    if (oR == ORI_ANY) oR = oL;
    const int o = x->side == 0 ? oL : oR;               /* the outer child's orientation */
    sym_merge(s, x, &L, oL, &R, oR, o, 1);
    return o;
}

/* lazy = 0: Geckosort1, 1: Squidsort1; floor(n/2) buffer slots as Frogsort1.
 * counters (may be NULL): [0] setup moves, [1] merge moves (including the
 * final reversal), [2] comparisons.  Returns 0, or -1 on allocation failure. */
int orc_symsort(uint64_t* keys, uint32_t* payload, int64_t n, int key_type, int order, int lazy,
                int64_t* counters)
{
    int64_t setup_moves = 0;
    sym_run s;
    memset(&s, 0, sizeof(s));
    s.f.c.key_type = key_type; s.f.c.order = order; s.f.g = 1; s.lazy = lazy ? 1 : 0;
    if (n >= 2) {
        int64_t b = n / 2, m = n + b;
        s.f.k = (uint64_t*)malloc((size_t)m * sizeof(uint64_t));
        s.f.p = payload ? (uint32_t*)malloc((size_t)m * sizeof(uint32_t)) : NULL;
        int64_t* dest = (int64_t*)malloc((size_t)n * sizeof(int64_t));
        if (!s.f.k || (payload && !s.f.p) || !dest) { free(s.f.k); free(s.f.p); free(dest); return -1; }
        memcpy(s.f.k, keys, (size_t)n * sizeof(uint64_t));
        if (payload) memcpy(s.f.p, payload, (size_t)n * sizeof(uint32_t));
        frog_node root = frog_root(n, 1);
        frog_setup_dest(&root, 1, dest);
        for (int64_t e = n - 1; e >= 0; e--) {          /* dest >= source, increasing: top down */
            if (dest[e] != e) {
                s.f.k[dest[e]] = s.f.k[e];
                if (payload) s.f.p[dest[e]] = s.f.p[e];
                setup_moves++;
            }
        }
        free(dest);
        if (sym_rec(&s, &root) == ORI_DESC) {           /* the root is data-left: slots [0, n) */
            for (int64_t i = 0, j = n - 1; i < j; i++, j--) {
                uint64_t tk = s.f.k[i]; s.f.k[i] = s.f.k[j]; s.f.k[j] = tk;
                if (payload) { uint32_t tp = s.f.p[i]; s.f.p[i] = s.f.p[j]; s.f.p[j] = tp; }
                s.f.c.moves += 2;
            }
        }
        memcpy(keys, s.f.k, (size_t)n * sizeof(uint64_t));
        if (payload) memcpy(payload, s.f.p, (size_t)n * sizeof(uint32_t));
        free(s.f.k); free(s.f.p);
    }
    if (counters) { counters[0] = setup_moves; counters[1] = s.f.c.moves; counters[2] = s.f.c.compares; }
    return 0;
}
