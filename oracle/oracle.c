/*
 * CPU oracle for batched 2-D distance reporting along a recursive space-filling curve
 * ("Simpler is Faster", arXiv 2508.19891).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct statement of
 * what the GPU path must compute.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load it.  It shares no code, header, table
 * or constant with the CUDA library, and the CUDA library never calls it.
 *
 * Conventions (the paper's notation, with the readings used throughout the project):
 *   - Domain D = [0, 2^w)^2 of integer points (the paper writes [1, 2^w], Sec. 2; the shift
 *     by one is immaterial).  The GPU path fixes w = 30; the oracle takes w as a parameter
 *     so that small grids can be enumerated exhaustively.
 *   - pi(p) is a bit string of length 2w, stored in the low 2w bits of a uint64.
 *   - Query (q, delta): integer centre q in D, integer radius delta >= 0.  The answer is the
 *     closed ball {i : (x_i - q_x)^2 + (y_i - q_y)^2 <= delta^2} (problem statement, Sec. 2),
 *     evaluated exactly in int64.
 *
 * Every function below cites the passage it follows.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORACLE_CURVE_Z 0
#define ORACLE_CURVE_HILBERT 1

/* ------------------------------------------------------------------------------------ */
/* Keys.                                                                                 */
/* ------------------------------------------------------------------------------------ */

/* Z-curve (Morton) key, Alg. 2: bit 2i of the output is bit i of x, bit 2i+1 is bit i of y,
 * for i in [w].  Written as the literal per-bit loop of the algorithm. */
uint64_t oracle_key_z(uint32_t x, uint32_t y, int w)
{
    uint64_t out = 0;
    for (int i = 0; i < w; ++i) {
        uint64_t xi = (x >> i) & 1u;
        uint64_t yi = (y >> i) & 1u;
        out |= xi << (2 * i);
        out |= yi << (2 * i + 1);
    }
    return out;
}

/* Hilbert key as a recursive space-filling curve (Sec. 2.1, "Choice of RSFC"; Def. 2.3).
 * Orientation (the paper does not fix one): the order-1 curve visits
 * (0,0) -> (0,1) -> (1,1) -> (1,0), i.e. the four quadrants get the 2-bit labels
 * lower-left 00, upper-left 01, upper-right 10, lower-right 11 (Lemma 1 assigns suffixes
 * 00,01,10,11 in visiting order).  Inside a quadrant the sub-square is mapped back to the
 * base orientation before its own quadrant is read:
 *   upper quadrants: unchanged;
 *   lower-left:  reflected in the main diagonal (x and y exchanged);
 *   lower-right: reflected in the anti-diagonal (x -> s-1-y, y -> s-1-x).
 * The label of the parent is a prefix of the label of each child, as Def. 2.3 requires. */
uint64_t oracle_key_h(uint32_t x, uint32_t y, int w)
{
    uint64_t key = 0;
    uint64_t xx = x, yy = y;
    for (int level = w - 1; level >= 0; --level) {
        uint64_t s = (uint64_t)1 << level;           /* side of the sub-square */
        int rx = (int)((xx >> level) & 1u);
        int ry = (int)((yy >> level) & 1u);
        int digit;
        if (!rx && !ry) digit = 0;      /* lower-left  */
        else if (!rx && ry) digit = 1;  /* upper-left  */
        else if (rx && ry) digit = 2;   /* upper-right */
        else digit = 3;                 /* lower-right */
        key = (key << 2) | (uint64_t)digit;
        /* coordinates inside the chosen sub-square */
        xx &= s - 1;
        yy &= s - 1;
        if (!ry) {
            if (rx) {   /* anti-diagonal reflection = point reflection followed by a swap */
                xx = (s - 1) - xx;
                yy = (s - 1) - yy;
            }
            uint64_t t = xx; xx = yy; yy = t;
        }
    }
    return key;
}

uint64_t oracle_key(uint32_t x, uint32_t y, int w, int curve)
{
    return curve == ORACLE_CURVE_HILBERT ? oracle_key_h(x, y, w) : oracle_key_z(x, y, w);
}

/* pi(p) for every input point (Sec. 3.1.1: "compute the bit strings pi(A[i])"). */
void oracle_keys(const int32_t* xy, uint64_t n, int w, int curve, uint64_t* keys)
{
    for (uint64_t i = 0; i < n; ++i)
        keys[i] = oracle_key((uint32_t)xy[2 * i], (uint32_t)xy[2 * i + 1], w, curve);
}

/* ------------------------------------------------------------------------------------ */
/* Construction: sort the points once by pi (Sec. 2, "store P in an array sorted by pi";  */
/* Sec. 3.1.1).  Ties are broken by input index, which makes the order total.             */
/* ------------------------------------------------------------------------------------ */

typedef struct { uint64_t key; uint32_t id; } oracle_pair;

static int pair_cmp(const void* a, const void* b)
{
    const oracle_pair* pa = (const oracle_pair*)a;
    const oracle_pair* pb = (const oracle_pair*)b;
    if (pa->key != pb->key) return pa->key < pb->key ? -1 : 1;
    if (pa->id != pb->id) return pa->id < pb->id ? -1 : 1;
    return 0;
}

/* Sort (key, id) pairs by key then id with the C library's qsort.
 * Outputs: sorted keys, the input index of each sorted entry, and its coordinates. */
int oracle_build(const int32_t* xy, uint64_t n, int w, int curve,
                 uint64_t* skeys, uint32_t* sids, int32_t* sxy)
{
    oracle_pair* pairs = (oracle_pair*)malloc((n ? n : 1) * sizeof(oracle_pair));
    if (!pairs) return -2;
    for (uint64_t i = 0; i < n; ++i) {
        pairs[i].key = oracle_key((uint32_t)xy[2 * i], (uint32_t)xy[2 * i + 1], w, curve);
        pairs[i].id = (uint32_t)i;
    }
    qsort(pairs, n, sizeof(oracle_pair), pair_cmp);
    for (uint64_t i = 0; i < n; ++i) {
        skeys[i] = pairs[i].key;
        sids[i] = pairs[i].id;
        sxy[2 * i] = xy[2 * (uint64_t)pairs[i].id];
        sxy[2 * i + 1] = xy[2 * (uint64_t)pairs[i].id + 1];
    }
    free(pairs);
    return 0;
}

/* A_P.lower_bound (Alg. 1): first index x with keys[x] >= t, or n. */
uint64_t oracle_lower_bound(const uint64_t* keys, uint64_t n, uint64_t t)
{
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (keys[mid] < t) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* ------------------------------------------------------------------------------------ */
/* cells(Q) (definition before Alg. 1) and the key interval of a cell (Observation).      */
/* ------------------------------------------------------------------------------------ */

/* Level l of the cells for a query radius delta: |.| is the side length, Q has side
 * 2*delta, and cells(Q) takes the cells C with |Q| <= |C| < 2|Q|, i.e. the level l with
 * 2*delta <= 2^l < 4*delta.  delta = 0 (Q is one point) takes the unit cells (l = 0).
 * A level above w would be larger than the domain; it is capped at w. */
int oracle_level(int64_t delta, int w)
{
    if (delta <= 0) return 0;
    int l = 0;
    while (((int64_t)1 << l) < 2 * delta) ++l;
    return l < w ? l : w;
}

/* Writes the key intervals [lo, hi] of cells(Q) for Q = [q - delta, q + delta]^2 clipped
 * to D, sorted by lo; returns how many (at most 4).  For a cell C at level l with lower-left
 * grid point c, pi(C) is the common 2(w - l)-bit prefix of its points (Def. 2.3), so
 * pi(C)o0 = (pi(c) >> 2l) << 2l and pi(C)o1 = pi(C)o0 + 4^l - 1 (Observation). */
int oracle_cells(int32_t qx, int32_t qy, int32_t delta, int w, int curve,
                 uint64_t lo[4], uint64_t hi[4], int* level_out)
{
    int64_t side = (int64_t)1 << w;
    int64_t d = delta;
    int64_t x0 = (int64_t)qx - d, x1 = (int64_t)qx + d;
    int64_t y0 = (int64_t)qy - d, y1 = (int64_t)qy + d;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > side - 1) x1 = side - 1;
    if (y1 > side - 1) y1 = side - 1;
    int l = oracle_level(d, w);
    if (level_out) *level_out = l;
    int cnt = 0;
    for (int64_t cy = y0 >> l; cy <= (y1 >> l); ++cy) {
        for (int64_t cx = x0 >> l; cx <= (x1 >> l); ++cx) {
            if (cnt == 4) return -1;   /* cannot happen: at most two cells per axis */
            uint64_t corner = oracle_key((uint32_t)(cx << l), (uint32_t)(cy << l), w, curve);
            uint64_t base = (l >= 32) ? 0 : ((corner >> (2 * l)) << (2 * l));
            uint64_t span = (l >= 32) ? ~(uint64_t)0 : (((uint64_t)1 << (2 * l)) - 1);
            lo[cnt] = base;
            hi[cnt] = base + span;
            ++cnt;
        }
    }
    /* sort by lo (insertion sort of at most four entries) */
    for (int i = 1; i < cnt; ++i) {
        uint64_t a = lo[i], b = hi[i];
        int j = i - 1;
        while (j >= 0 && lo[j] > a) { lo[j + 1] = lo[j]; hi[j + 1] = hi[j]; --j; }
        lo[j + 1] = a; hi[j + 1] = b;
    }
    return cnt;
}

/* The query's window: the closed disc dx^2 + dy^2 <= delta^2 of the problem statement (norm 0),
 * or the closed square max(|dx|, |dy|) <= delta (norm 1), the axis-parallel window of side
 * 2 delta + 1 points that the experiments of Sec. 3 query (their windows are squares; the
 * result sizes printed in App. B match a square, not a disc). */
static int in_window(int64_t dx, int64_t dy, int64_t delta, int norm)
{
    if (norm == 1) return (dx < 0 ? -dx : dx) <= delta && (dy < 0 ? -dy : dy) <= delta;
    return dx * dx + dy * dy <= delta * delta;
}

/* Refined cover (a finer quadtree level than cells(Q), Sec. 2 "Efficiency" notes the cover's
 * volume can be 2 * 2^d times that of Q): the cells at level l' = max(0, l - drop), where l is
 * the level of cells(Q), that contain at least one integer point of the closed ball
 * B_delta(q) within the domain -- of the window of `norm` (in_window): for the square window
 * every cell meeting the clipped square Q qualifies; returns how many (at most
 * (2^drop + 1)^2), key intervals sorted by lo, not merged.  drop = 0 keeps only cells(Q)'s
 * cells that meet the window. */
int oracle_cells_refined_norm(int32_t qx, int32_t qy, int32_t delta, int w, int curve, int drop, int norm,
                              uint64_t* lo, uint64_t* hi, int maxc)
{
    int64_t side = (int64_t)1 << w;
    int64_t d = delta;
    int64_t x0 = (int64_t)qx - d, x1 = (int64_t)qx + d;
    int64_t y0 = (int64_t)qy - d, y1 = (int64_t)qy + d;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > side - 1) x1 = side - 1;
    if (y1 > side - 1) y1 = side - 1;
    int l = oracle_level(d, w) - drop;
    if (l < 0) l = 0;
    int cnt = 0;
    for (int64_t cy = y0 >> l; cy <= (y1 >> l); ++cy) {
        for (int64_t cx = x0 >> l; cx <= (x1 >> l); ++cx) {
            /* nearest integer point of the cell to q */
            int64_t ax0 = cx << l, ax1 = ((cx + 1) << l) - 1;
            int64_t ay0 = cy << l, ay1 = ((cy + 1) << l) - 1;
            int64_t dx = 0, dy = 0;
            if (qx < ax0) dx = ax0 - qx; else if (qx > ax1) dx = qx - ax1;
            if (qy < ay0) dy = ay0 - qy; else if (qy > ay1) dy = qy - ay1;
            if (!in_window(dx, dy, d, norm)) continue;
            if (cnt == maxc) return -1;
            uint64_t corner = oracle_key((uint32_t)(cx << l), (uint32_t)(cy << l), w, curve);
            uint64_t span = ((uint64_t)1 << (2 * l)) - 1;
            lo[cnt] = (corner >> (2 * l)) << (2 * l);
            hi[cnt] = lo[cnt] + span;
            ++cnt;
        }
    }
    for (int i = 1; i < cnt; ++i) {
        uint64_t a = lo[i], b = hi[i];
        int j = i - 1;
        while (j >= 0 && lo[j] > a) { lo[j + 1] = lo[j]; hi[j + 1] = hi[j]; --j; }
        lo[j + 1] = a; hi[j + 1] = b;
    }
    return cnt;
}

int oracle_cells_refined(int32_t qx, int32_t qy, int32_t delta, int w, int curve, int drop,
                         uint64_t* lo, uint64_t* hi, int maxc)
{
    return oracle_cells_refined_norm(qx, qy, delta, w, curve, drop, 0, lo, hi, maxc);
}

/* ------------------------------------------------------------------------------------ */
/* Query, Alg. 1: for each cell (in key order) lower_bound the start of its interval, scan */
/* while the key is <= pi(C)o1 (inclusive end, Observation), and report every point with  */
/* squared distance <= delta^2 (closed ball of the problem statement).                      */
/* ------------------------------------------------------------------------------------ */

static int query_valid(int32_t qx, int32_t qy, int32_t delta, int w)
{
    int64_t side = (int64_t)1 << w;
    return qx >= 0 && qy >= 0 && (int64_t)qx < side && (int64_t)qy < side && delta >= 0;
}

/* Reports the hits of one query; writes them to out (if not NULL) and returns the count.
 * scanned (if not NULL) receives the number of array entries visited. */
static uint64_t query_one(const uint64_t* skeys, const uint32_t* sids, const int32_t* sxy,
                          uint64_t n, int32_t qx, int32_t qy, int32_t delta, int w, int curve,
                          int norm, uint32_t* out, uint64_t* scanned)
{
    if (!query_valid(qx, qy, delta, w)) { if (scanned) *scanned = 0; return 0; }
    uint64_t lo[4], hi[4];
    int cnt = oracle_cells(qx, qy, delta, w, curve, lo, hi, NULL);
    uint64_t k = 0, s = 0;
    for (int c = 0; c < cnt; ++c) {
        uint64_t x = oracle_lower_bound(skeys, n, lo[c]);
        while (x < n && skeys[x] <= hi[c]) {
            int64_t dx = (int64_t)sxy[2 * x] - qx;
            int64_t dy = (int64_t)sxy[2 * x + 1] - qy;
            if (in_window(dx, dy, delta, norm)) {
                if (out) out[k] = sids[x];
                ++k;
            }
            ++x;
            ++s;
        }
    }
    if (scanned) *scanned = s;
    return k;
}

typedef struct {
    const uint64_t* skeys; const uint32_t* sids; const int32_t* sxy; uint64_t n;
    const int32_t* q; const int32_t* delta; uint64_t m0, m1; int w, curve, norm;
    uint64_t* counts; const uint64_t* offsets; uint32_t* out_ids; uint64_t* scanned;
} query_job;

static void* query_worker(void* arg)
{
    query_job* j = (query_job*)arg;
    for (uint64_t i = j->m0; i < j->m1; ++i) {
        uint32_t* out = j->out_ids ? j->out_ids + j->offsets[i] : NULL;
        uint64_t s = 0;
        uint64_t k = query_one(j->skeys, j->sids, j->sxy, j->n, j->q[2 * i], j->q[2 * i + 1],
                               j->delta[i], j->w, j->curve, j->norm, out, &s);
        if (j->counts) j->counts[i] = k;
        if (j->scanned) j->scanned[i] = s;
    }
    return NULL;
}

/* Runs the queries [0, m) on `threads` host threads, each taking a contiguous block of
 * queries.  With out_ids == NULL only counts (and scanned) are produced; otherwise the ids of
 * query i are written at out_ids[offsets[i] ...].  Queries are independent, so the split
 * does not change any result. */
int oracle_query_norm(const uint64_t* skeys, const uint32_t* sids, const int32_t* sxy, uint64_t n,
                      const int32_t* q, const int32_t* delta, uint64_t m, int w, int curve, int norm,
                      uint64_t* counts, const uint64_t* offsets, uint32_t* out_ids,
                      uint64_t* scanned, int threads)
{
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > m) threads = (int)(m ? m : 1);
    query_job* jobs = (query_job*)calloc((size_t)threads, sizeof(query_job));
    pthread_t* tids = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tids) { free(jobs); free(tids); return -2; }
    for (int t = 0; t < threads; ++t) {
        query_job* j = &jobs[t];
        j->skeys = skeys; j->sids = sids; j->sxy = sxy; j->n = n;
        j->q = q; j->delta = delta; j->w = w; j->curve = curve; j->norm = norm;
        j->m0 = m * (uint64_t)t / (uint64_t)threads;
        j->m1 = m * (uint64_t)(t + 1) / (uint64_t)threads;
        j->counts = counts; j->offsets = offsets; j->out_ids = out_ids; j->scanned = scanned;
    }
    if (threads == 1) {
        query_worker(&jobs[0]);
    } else {
        for (int t = 0; t < threads; ++t) pthread_create(&tids[t], NULL, query_worker, &jobs[t]);
        for (int t = 0; t < threads; ++t) pthread_join(tids[t], NULL);
    }
    free(jobs);
    free(tids);
    return 0;
}

/* Alg. 1 with the disc of the problem statement. */
int oracle_query(const uint64_t* skeys, const uint32_t* sids, const int32_t* sxy, uint64_t n,
                 const int32_t* q, const int32_t* delta, uint64_t m, int w, int curve,
                 uint64_t* counts, const uint64_t* offsets, uint32_t* out_ids,
                 uint64_t* scanned, int threads)
{
    return oracle_query_norm(skeys, sids, sxy, n, q, delta, m, w, curve, 0, counts, offsets, out_ids,
                             scanned, threads);
}

/* ------------------------------------------------------------------------------------ */
/* Brute force over the unsorted input: the problem statement of Sec. 2 taken literally.  */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    const int32_t* xy; uint64_t n; const int32_t* q; const int32_t* delta;
    uint64_t m0, m1; int w, norm; uint64_t* counts; const uint64_t* offsets; uint32_t* out_ids;
} brute_job;

static void* brute_worker(void* arg)
{
    brute_job* j = (brute_job*)arg;
    for (uint64_t i = j->m0; i < j->m1; ++i) {
        int32_t qx = j->q[2 * i], qy = j->q[2 * i + 1], dl = j->delta[i];
        uint64_t k = 0;
        if (query_valid(qx, qy, dl, j->w)) {
            for (uint64_t p = 0; p < j->n; ++p) {
                int64_t dx = (int64_t)j->xy[2 * p] - qx;
                int64_t dy = (int64_t)j->xy[2 * p + 1] - qy;
                if (in_window(dx, dy, dl, j->norm)) {
                    if (j->out_ids) j->out_ids[j->offsets[i] + k] = (uint32_t)p;
                    ++k;
                }
            }
        }
        if (j->counts) j->counts[i] = k;
    }
    return NULL;
}

/* Per-query hits in ascending input index (not key) order. */
int oracle_brute_norm(const int32_t* xy, uint64_t n, const int32_t* q, const int32_t* delta,
                      uint64_t m, int w, int norm, uint64_t* counts, const uint64_t* offsets,
                      uint32_t* out_ids, int threads)
{
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > m) threads = (int)(m ? m : 1);
    brute_job* jobs = (brute_job*)calloc((size_t)threads, sizeof(brute_job));
    pthread_t* tids = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tids) { free(jobs); free(tids); return -2; }
    for (int t = 0; t < threads; ++t) {
        brute_job* j = &jobs[t];
        j->xy = xy; j->n = n; j->q = q; j->delta = delta; j->w = w; j->norm = norm;
        j->m0 = m * (uint64_t)t / (uint64_t)threads;
        j->m1 = m * (uint64_t)(t + 1) / (uint64_t)threads;
        j->counts = counts; j->offsets = offsets; j->out_ids = out_ids;
    }
    if (threads == 1) {
        brute_worker(&jobs[0]);
    } else {
        for (int t = 0; t < threads; ++t) pthread_create(&tids[t], NULL, brute_worker, &jobs[t]);
        for (int t = 0; t < threads; ++t) pthread_join(tids[t], NULL);
    }
    free(jobs);
    free(tids);
    return 0;
}

int oracle_brute(const int32_t* xy, uint64_t n, const int32_t* q, const int32_t* delta,
                 uint64_t m, int w, uint64_t* counts, const uint64_t* offsets,
                 uint32_t* out_ids, int threads)
{
    return oracle_brute_norm(xy, n, q, delta, m, w, 0, counts, offsets, out_ids, threads);
}

/* ------------------------------------------------------------------------------------ */
/* Early-termination quadtree (Sec. 2.2, "Early termination").                           */
/* ------------------------------------------------------------------------------------ */

/* The boolean of every node of the complete quadtree of depth D over the bounding box G =
 * [0, 2^w)^2: node v at depth t (0 <= t <= D) is the cell of level w - t whose label (the
 * key prefix of Def. 2.3) is v; its boolean is true iff the cell contains a point.  Stored
 * one bit per node, depth after depth: depth t starts at bit (4^t - 1) / 3, node v at that
 * start + v.  Written as the definition: every point marks its cell on every level.
 * `bits` must hold ((4^(D+1) - 1) / 3 + 31) / 32 words; it is cleared first. */
void oracle_occupancy(const uint64_t* keys, uint64_t n, int w, int D, uint32_t* bits)
{
    const uint64_t total = (((uint64_t)1 << (2 * (D + 1))) - 1) / 3;
    memset(bits, 0, ((total + 31) / 32) * sizeof(uint32_t));
    for (uint64_t i = 0; i < n; ++i) {
        for (int t = 0; t <= D; ++t) {
            const uint64_t start = (((uint64_t)1 << (2 * t)) - 1) / 3;
            const uint64_t v = keys[i] >> (2 * (w - t));
            const uint64_t b = start + v;
            bits[b / 32] |= 1u << (b % 32);
        }
    }
}

/* Whether the cell of level l whose key interval starts at `lo` may hold a point by the
 * early-termination quadtree of depth D: the cell's own node when it is at depth <= D, else
 * its ancestor at depth D (which only answers "empty" for the whole ancestor). */
int oracle_cell_occupied(const uint32_t* bits, int w, int D, int l, uint64_t lo)
{
    int t = w - l;
    if (t > D) t = D;
    const uint64_t start = (((uint64_t)1 << (2 * t)) - 1) / 3;
    const uint64_t b = start + (lo >> (2 * (w - t)));
    return (int)((bits[b / 32] >> (b % 32)) & 1u);
}

/* ------------------------------------------------------------------------------------ */
/* d = 3: the Z curve in Z^3 (the paper notes its Z implementation extends to R^d,       */
/* Sec. 2.1; cells(Q) then has at most 2^d = 8 cells, Sec. 1.2).                         */
/* Domain [0, 2^w)^3; pi(p) has 3w bits: bit 3i = x_i, bit 3i+1 = y_i, bit 3i+2 = z_i     */
/* (Alg. 2 with a third interleaved coordinate).  The GPU path fixes w = 21 (63 bits).   */
/* ------------------------------------------------------------------------------------ */

/* Z key in 3-D, the literal per-bit loop. */
uint64_t oracle_key_z3(uint32_t x, uint32_t y, uint32_t z, int w)
{
    uint64_t out = 0;
    for (int i = 0; i < w; ++i) {
        out |= (uint64_t)((x >> i) & 1u) << (3 * i);
        out |= (uint64_t)((y >> i) & 1u) << (3 * i + 1);
        out |= (uint64_t)((z >> i) & 1u) << (3 * i + 2);
    }
    return out;
}

/* Sorted array of 3-D points: keys, input indices and coordinates sorted by (key, id). */
int oracle_build3(const int32_t* xyz, uint64_t n, int w, uint64_t* skeys, uint32_t* sids, int32_t* sxyz)
{
    oracle_pair* pairs = (oracle_pair*)malloc((n ? n : 1) * sizeof(oracle_pair));
    if (!pairs) return -2;
    for (uint64_t i = 0; i < n; ++i) {
        pairs[i].key = oracle_key_z3((uint32_t)xyz[3 * i], (uint32_t)xyz[3 * i + 1], (uint32_t)xyz[3 * i + 2], w);
        pairs[i].id = (uint32_t)i;
    }
    qsort(pairs, n, sizeof(oracle_pair), pair_cmp);
    for (uint64_t i = 0; i < n; ++i) {
        skeys[i] = pairs[i].key;
        sids[i] = pairs[i].id;
        for (int c = 0; c < 3; ++c) sxyz[3 * i + c] = xyz[3 * (uint64_t)pairs[i].id + c];
    }
    free(pairs);
    return 0;
}

/* cells(Q) in 3-D: Q = [q - delta, q + delta]^3 clipped to the domain, level l as in 2-D
 * (side 2^l with 2 delta <= 2^l < 4 delta, capped at w), the cells of that level meeting Q
 * (at most two per axis, so at most 8), each with the key interval [pi(C)o0, pi(C)o1] of
 * length 8^l; sorted by lo. */
int oracle_cells3(int32_t qx, int32_t qy, int32_t qz, int32_t delta, int w, uint64_t lo[8], uint64_t hi[8],
                  int* level_out)
{
    const int64_t side = (int64_t)1 << w;
    const int64_t d = delta;
    int64_t a0[3], a1[3];
    const int64_t c[3] = {qx, qy, qz};
    for (int k = 0; k < 3; ++k) {
        a0[k] = c[k] - d < 0 ? 0 : c[k] - d;
        a1[k] = c[k] + d > side - 1 ? side - 1 : c[k] + d;
    }
    const int l = oracle_level(d, w);
    if (level_out) *level_out = l;
    int cnt = 0;
    for (int64_t cz = a0[2] >> l; cz <= (a1[2] >> l); ++cz)
        for (int64_t cy = a0[1] >> l; cy <= (a1[1] >> l); ++cy)
            for (int64_t cx = a0[0] >> l; cx <= (a1[0] >> l); ++cx) {
                if (cnt == 8) return -1;   /* cannot happen: at most two cells per axis */
                const uint64_t corner = oracle_key_z3((uint32_t)(cx << l), (uint32_t)(cy << l), (uint32_t)(cz << l), w);
                const uint64_t span = (3 * l >= 64) ? ~(uint64_t)0 : (((uint64_t)1 << (3 * l)) - 1);
                lo[cnt] = corner & ~span;
                hi[cnt] = lo[cnt] + span;
                ++cnt;
            }
    for (int i = 1; i < cnt; ++i) {
        const uint64_t a = lo[i], b = hi[i];
        int j = i - 1;
        while (j >= 0 && lo[j] > a) { lo[j + 1] = lo[j]; hi[j + 1] = hi[j]; --j; }
        lo[j + 1] = a; hi[j + 1] = b;
    }
    return cnt;
}

static int query3_valid(int32_t qx, int32_t qy, int32_t qz, int32_t delta, int w)
{
    const int64_t side = (int64_t)1 << w;
    return qx >= 0 && qy >= 0 && qz >= 0 && qx < side && qy < side && qz < side && delta >= 0;
}

/* Alg. 1 in 3-D for queries [m0, m1): closed ball dx^2 + dy^2 + dz^2 <= delta^2 in int64. */
static uint64_t query3_one(const uint64_t* skeys, const uint32_t* sids, const int32_t* sxyz, uint64_t n,
                           const int32_t* q, int32_t delta, int w, uint32_t* out)
{
    if (!query3_valid(q[0], q[1], q[2], delta, w)) return 0;
    uint64_t lo[8], hi[8];
    const int cnt = oracle_cells3(q[0], q[1], q[2], delta, w, lo, hi, NULL);
    const int64_t d2 = (int64_t)delta * delta;
    uint64_t k = 0;
    for (int c = 0; c < cnt; ++c) {
        for (uint64_t x = oracle_lower_bound(skeys, n, lo[c]); x < n && skeys[x] <= hi[c]; ++x) {
            const int64_t dx = (int64_t)sxyz[3 * x] - q[0];
            const int64_t dy = (int64_t)sxyz[3 * x + 1] - q[1];
            const int64_t dz = (int64_t)sxyz[3 * x + 2] - q[2];
            if (dx * dx + dy * dy + dz * dz <= d2) {
                if (out) out[k] = sids[x];
                ++k;
            }
        }
    }
    return k;
}

/* Counts (offsets == NULL) or ids (written at out_ids + offsets[i]) of every query, one thread. */
int oracle_query3(const uint64_t* skeys, const uint32_t* sids, const int32_t* sxyz, uint64_t n,
                  const int32_t* q, const int32_t* delta, uint64_t m, int w, uint64_t* counts,
                  const uint64_t* offsets, uint32_t* out_ids)
{
    for (uint64_t i = 0; i < m; ++i) {
        const uint64_t k = query3_one(skeys, sids, sxyz, n, q + 3 * i, delta[i], w,
                                      out_ids ? out_ids + offsets[i] : NULL);
        if (counts) counts[i] = k;
    }
    return 0;
}

/* Brute force in 3-D: ids ascending per query. */
int oracle_brute3(const int32_t* xyz, uint64_t n, const int32_t* q, const int32_t* delta, uint64_t m, int w,
                  uint64_t* counts, const uint64_t* offsets, uint32_t* out_ids)
{
    for (uint64_t i = 0; i < m; ++i) {
        uint64_t k = 0;
        if (query3_valid(q[3 * i], q[3 * i + 1], q[3 * i + 2], delta[i], w)) {
            const int64_t d2 = (int64_t)delta[i] * delta[i];
            for (uint64_t p = 0; p < n; ++p) {
                const int64_t dx = (int64_t)xyz[3 * p] - q[3 * i];
                const int64_t dy = (int64_t)xyz[3 * p + 1] - q[3 * i + 1];
                const int64_t dz = (int64_t)xyz[3 * p + 2] - q[3 * i + 2];
                if (dx * dx + dy * dy + dz * dz <= d2) {
                    if (out_ids) out_ids[offsets[i] + k] = (uint32_t)p;
                    ++k;
                }
            }
        }
        if (counts) counts[i] = k;
    }
    return 0;
}

/* Refined 3-D cover (as oracle_cells_refined in 2-D): the cells of level max(0, l - drop)
 * that contain an integer point of the closed ball (the distance from q to the cell's
 * nearest integer point is at most delta), at most (2^drop + 1)^3; sorted by lo, not merged.
 * Returns -1 if more than maxc. */
int oracle_cells3_refined(int32_t qx, int32_t qy, int32_t qz, int32_t delta, int w, int drop, uint64_t* lo,
                          uint64_t* hi, int maxc)
{
    const int64_t side = (int64_t)1 << w;
    const int64_t d = delta;
    const int64_t c[3] = {qx, qy, qz};
    int64_t a0[3], a1[3];
    for (int k = 0; k < 3; ++k) {
        a0[k] = c[k] - d < 0 ? 0 : c[k] - d;
        a1[k] = c[k] + d > side - 1 ? side - 1 : c[k] + d;
    }
    int l = oracle_level(d, w) - drop;
    if (l < 0) l = 0;
    int cnt = 0;
    for (int64_t cz = a0[2] >> l; cz <= (a1[2] >> l); ++cz)
        for (int64_t cy = a0[1] >> l; cy <= (a1[1] >> l); ++cy)
            for (int64_t cx = a0[0] >> l; cx <= (a1[0] >> l); ++cx) {
                const int64_t cc[3] = {cx, cy, cz};
                int64_t dist2 = 0;
                for (int k = 0; k < 3; ++k) {
                    const int64_t b0 = cc[k] << l, b1 = ((cc[k] + 1) << l) - 1;
                    const int64_t e = c[k] < b0 ? b0 - c[k] : (c[k] > b1 ? c[k] - b1 : 0);
                    dist2 += e * e;
                }
                if (dist2 > d * d) continue;
                if (cnt == maxc) return -1;
                const uint64_t corner = oracle_key_z3((uint32_t)(cx << l), (uint32_t)(cy << l), (uint32_t)(cz << l), w);
                const uint64_t span = (3 * l >= 64) ? ~(uint64_t)0 : (((uint64_t)1 << (3 * l)) - 1);
                lo[cnt] = corner & ~span;
                hi[cnt] = lo[cnt] + span;
                ++cnt;
            }
    for (int i = 1; i < cnt; ++i) {
        const uint64_t a = lo[i], b = hi[i];
        int j = i - 1;
        while (j >= 0 && lo[j] > a) { lo[j + 1] = lo[j]; hi[j + 1] = hi[j]; --j; }
        lo[j + 1] = a; hi[j + 1] = b;
    }
    return cnt;
}
