/*
 * graphgen.c -- seeded synthetic graph generators (inputs only).
 *
 * This file draws random graphs and turns edge lists into a symmetric,
 * deduplicated CSR. It holds none of the triangle-counting arithmetic: no
 * orientation, no intersection, no counting. Both the CPU oracle's tests and
 * the GPU path's tests/bench take their inputs from here, and from nowhere
 * else.
 *
 * Randomness: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014). A stream is a 64-bit key; draw k of the
 * stream is mix(key + (k+1)*gamma), which is exactly the k-th output of a
 * SplitMix64 generator started at state = key, so any draw can be computed
 * independently (counter-based use).
 *
 * Determinism across machines: only IEEE-exact operations (+ - * / sqrt,
 * conversions) touch floating point, and the file is compiled with
 * -ffp-contract=off, so x86-64 and aarch64 produce the same graphs. The one
 * transcendental that ER skipping needs (log) and the one that the batched
 * size draw needs (2^x) are computed below from their series with basic
 * operations only, instead of calling libm, whose last bits may differ between
 * platforms.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Key of stream `stream` under `seed` (e.g. stream = graph index in a batch). */
uint64_t gg_stream_key(uint64_t seed, uint64_t stream) {
    return mix64(mix64(seed + GG_GAMMA) ^ mix64((stream + 1) * 0xD1B54A32D192ED03ULL));
}

/* Draw k of stream `key`. */
uint64_t gg_draw(uint64_t key, uint64_t k) { return mix64(key + (k + 1) * GG_GAMMA); }

/* Uniform double in [0,1) from the top 53 bits. */
static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

double gg_u01(uint64_t key, uint64_t k) { return u01(gg_draw(key, k)); }

/* ---------- deterministic log / exp2 (series; basic operations only) ---------- */

static const double GG_LN2 = 0.69314718055994530942;
static const double GG_SQRT2 = 1.41421356237309504880;

/* Natural log of x > 0: x = m * 2^e with m in [sqrt(1/2), sqrt(2)); then
 * log m = 2 * atanh(s), s = (m-1)/(m+1), |s| < 0.1716, summed to 1e-17. */
double gg_log(double x) {
    if (!(x > 0.0)) return -1.0e308;
    int e = 0;
    while (x >= GG_SQRT2) { x *= 0.5; e++; }
    while (x < GG_SQRT2 * 0.5) { x *= 2.0; e--; }
    double s = (x - 1.0) / (x + 1.0), s2 = s * s, term = s, sum = 0.0;
    for (int k = 1; k < 60; k += 2) { sum += term / (double)k; term *= s2; }
    return 2.0 * sum + (double)e * GG_LN2;
}

/* 2^f for f in [0, 16): integer part by doubling, fraction by the exp series. */
double gg_exp2(double f) {
    int ip = (int)f;
    double fr = (f - (double)ip) * GG_LN2, term = 1.0, sum = 1.0;
    for (int k = 1; k < 30; k++) { term *= fr / (double)k; sum += term; }
    for (int i = 0; i < ip; i++) sum *= 2.0;
    return sum;
}

/* ---------- R-MAT (Chakrabarti, Zhan & Faloutsos, SDM 2004) ---------- */

/* Draw `ne` directed edges of an R-MAT graph on 2^scale vertices with quadrant
 * probabilities (a, b, c, 1-a-b-c), one level per bit, most significant first.
 * Edge e, attempt t, level l uses draw (e*64 + t)*64 + l of the stream. If
 * n_keep < 2^scale an edge with an endpoint >= n_keep is redrawn (up to 64
 * attempts; an edge that fails them all is written as the self-loop (0,0),
 * which CSR building drops). Self-loops and duplicates are left in; the CSR
 * builder removes them. */
void gg_rmat_edges(int scale, int64_t ne, double a, double b, double c, uint64_t key,
                   int64_t n_keep, int32_t* src, int32_t* dst) {
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; e++) {
        int64_t u = 0, v = 0;
        int ok = 0;
        for (int t = 0; t < 64 && !ok; t++) {
            u = 0; v = 0;
            uint64_t base = ((uint64_t)e * 64u + (uint64_t)t) * 64u;
            for (int l = 0; l < scale; l++) {
                double r = u01(gg_draw(key, base + (uint64_t)l));
                int bu = 0, bv = 0;
                if (r < a) { }
                else if (r < ab) { bv = 1; }
                else if (r < abc) { bu = 1; }
                else { bu = 1; bv = 1; }
                u = (u << 1) | bu;
                v = (v << 1) | bv;
            }
            ok = (u < n_keep && v < n_keep);
        }
        if (!ok) { u = 0; v = 0; }
        src[e] = (int32_t)u;
        dst[e] = (int32_t)v;
    }
}

/* ---------- Erdos-Renyi G(n, p) by geometric skipping ---------- */

/* Batagelj & Brandes, "Efficient generation of large random networks",
 * Phys. Rev. E 71 (2005), algorithm for G(n,p): walk the pairs (v, w), w < v,
 * in row order, jumping over a geometric number of absent pairs each time.
 * Writes at most `cap` edges; returns the number of edges of the graph (which
 * may exceed cap, in which case the caller retries with a larger buffer). */
int64_t gg_er_edges(int64_t n, double p, uint64_t key, int64_t cap, int32_t* src, int32_t* dst) {
    int64_t m = 0;
    if (n < 2 || p <= 0.0) return 0;
    if (p >= 1.0) {
        for (int64_t v = 1; v < n; v++)
            for (int64_t w = 0; w < v; w++) {
                if (m < cap) { src[m] = (int32_t)v; dst[m] = (int32_t)w; }
                m++;
            }
        return m;
    }
    const double lq = gg_log(1.0 - p);
    int64_t v = 1, w = -1;
    uint64_t k = 0;
    while (v < n) {
        double r = u01(gg_draw(key, k++));
        double skip = gg_log(1.0 - r) / lq;          /* >= 0 */
        if (skip > 4.0e18) skip = 4.0e18;
        w = w + 1 + (int64_t)skip;
        while (w >= v && v < n) { w -= v; v++; }
        if (v < n) {
            if (m < cap) { src[m] = (int32_t)v; dst[m] = (int32_t)w; }
            m++;
        }
    }
    return m;
}

/* ---------- random geometric graph in the unit square ---------- */

/* n points, coordinates x = draw 2i, y = draw 2i+1 of the stream, as uniform
 * doubles in [0,1). */
void gg_rgg_points(int64_t n, uint64_t key, double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        x[i] = u01(gg_draw(key, 2u * (uint64_t)i));
        y[i] = u01(gg_draw(key, 2u * (uint64_t)i + 1u));
    }
}

static void insertion_sort_i32(int32_t* a, int64_t len) {
    for (int64_t i = 1; i < len; i++) {
        int32_t k = a[i];
        int64_t j = i - 1;
        while (j >= 0 && a[j] > k) { a[j + 1] = a[j]; j--; }
        a[j + 1] = k;
    }
}

/* Edge {i,j} iff (xi-xj)^2 + (yi-yj)^2 < r^2 (no wrap-around). Uses a grid of
 * cells of side >= r, so only the 3x3 neighbouring cells are scanned.
 * Two-phase: with col == NULL, fills row_ptr (n+1, int64) and returns nnz;
 * with col != NULL (nnz entries, row_ptr from phase one), fills sorted rows.
 * Vertex ids are point indices (generation order). */
int64_t gg_rgg_csr(int64_t n, const double* x, const double* y, double r,
                   int64_t* row_ptr, int32_t* col) {
    int64_t g = (int64_t)(1.0 / r);
    if (g < 1) g = 1;
    if (g > 65536) g = 65536;
    const int64_t ncell = g * g;
    int64_t* cstart = (int64_t*)calloc((size_t)(ncell + 1), sizeof(int64_t));
    int32_t* cpts = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* pc = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!cstart || !cpts || !pc) { free(cstart); free(cpts); free(pc); return -1; }
    for (int64_t i = 0; i < n; i++) {
        int64_t cx = (int64_t)(x[i] * (double)g), cy = (int64_t)(y[i] * (double)g);
        if (cx >= g) cx = g - 1;
        if (cy >= g) cy = g - 1;
        pc[i] = (int32_t)(cy * g + cx);
        cstart[pc[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) cstart[c + 1] += cstart[c];
    {
        int64_t* cur = (int64_t*)malloc((size_t)ncell * sizeof(int64_t));
        memcpy(cur, cstart, (size_t)ncell * sizeof(int64_t));
        for (int64_t i = 0; i < n; i++) cpts[cur[pc[i]]++] = (int32_t)i;   /* ascending i per cell */
        free(cur);
    }
    const double r2 = r * r;
    const int fill = (col != NULL);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; i++) {
        int64_t c = pc[i], cx = c % g, cy = c / g, cnt = 0;
        int64_t base = fill ? row_ptr[i] : 0;
        for (int64_t dy = -1; dy <= 1; dy++) {
            int64_t yy = cy + dy;
            if (yy < 0 || yy >= g) continue;
            for (int64_t dx = -1; dx <= 1; dx++) {
                int64_t xx = cx + dx;
                if (xx < 0 || xx >= g) continue;
                int64_t cc = yy * g + xx;
                for (int64_t k = cstart[cc]; k < cstart[cc + 1]; k++) {
                    int32_t j = cpts[k];
                    if (j == i) continue;
                    double ddx = x[i] - x[j], ddy = y[i] - y[j];
                    if (ddx * ddx + ddy * ddy < r2) {
                        if (fill) col[base + cnt] = j;
                        cnt++;
                    }
                }
            }
        }
        if (fill) insertion_sort_i32(col + base, cnt);
        else row_ptr[i + 1] = cnt;
    }
    int64_t nnz = 0;
    if (!fill) {
        row_ptr[0] = 0;
        for (int64_t i = 0; i < n; i++) row_ptr[i + 1] += row_ptr[i];
    }
    nnz = row_ptr[n];
    free(cstart); free(cpts); free(pc);
    return nnz;
}

/* ---------- edge list -> symmetric, deduplicated, sorted CSR ---------- */

static void radix_sort_u32(uint32_t* a, uint32_t* tmp, int64_t len) {
    int64_t cnt[2048];
    uint32_t* s = a; uint32_t* d = tmp;
    for (int pass = 0; pass < 3; pass++) {
        int shift = pass * 11;
        memset(cnt, 0, sizeof(cnt));
        for (int64_t i = 0; i < len; i++) cnt[(s[i] >> shift) & 2047]++;
        int64_t acc = 0;
        for (int k = 0; k < 2048; k++) { int64_t t = cnt[k]; cnt[k] = acc; acc += t; }
        for (int64_t i = 0; i < len; i++) d[cnt[(s[i] >> shift) & 2047]++] = s[i];
        uint32_t* t = s; s = d; d = t;
    }
    if (s != a) memcpy(a, s, (size_t)len * sizeof(uint32_t));
}

/* Builds the CSR of the simple undirected graph spanned by the `ne` edges
 * (src[e], dst[e]): every edge is stored in both directions, self-loops and
 * edges with an endpoint outside [0, n) are dropped, duplicates are removed,
 * and every row is sorted ascending. row_ptr has n+1 entries; col must hold
 * 2*ne entries (the rows are compacted in place). Returns nnz (= 2 * number of
 * undirected edges), or -1 on allocation failure. */
int64_t gg_build_csr(int64_t n, int64_t ne, const int32_t* src, const int32_t* dst,
                     int64_t* row_ptr, int32_t* col) {
    int64_t* cur = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
    if (!cur) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; e++) {
        int64_t s = src[e], d = dst[e];
        if (s == d || s < 0 || d < 0 || s >= n || d >= n) continue;
        __atomic_fetch_add(&cur[s], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&cur[d], 1, __ATOMIC_RELAXED);
    }
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n; i++) row_ptr[i + 1] = row_ptr[i] + cur[i];
    memcpy(cur, row_ptr, (size_t)n * sizeof(int64_t));
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; e++) {
        int64_t s = src[e], d = dst[e];
        if (s == d || s < 0 || d < 0 || s >= n || d >= n) continue;
        col[__atomic_fetch_add(&cur[s], 1, __ATOMIC_RELAXED)] = (int32_t)d;
        col[__atomic_fetch_add(&cur[d], 1, __ATOMIC_RELAXED)] = (int32_t)s;
    }
    /* sort + unique each row; cur[i] := unique length */
#pragma omp parallel
    {
        int64_t tcap = 0;
        uint32_t* tmp = NULL;
#pragma omp for schedule(dynamic, 1024)
        for (int64_t i = 0; i < n; i++) {
            int64_t b = row_ptr[i], len = row_ptr[i + 1] - b;
            int32_t* r = col + b;
            if (len > 64) {
                if (len > tcap) { free(tmp); tcap = len; tmp = (uint32_t*)malloc((size_t)tcap * sizeof(uint32_t)); }
                radix_sort_u32((uint32_t*)r, tmp, len);
            } else {
                insertion_sort_i32(r, len);
            }
            int64_t k = 0;
            for (int64_t j = 0; j < len; j++)
                if (k == 0 || r[j] != r[k - 1]) r[k++] = r[j];
            cur[i] = k;
        }
        free(tmp);
    }
    int64_t w = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t b = row_ptr[i], len = cur[i];
        if (w != b) memmove(col + w, col + b, (size_t)len * sizeof(int32_t));
        row_ptr[i] = w;
        w += len;
    }
    row_ptr[n] = w;
    free(cur);
    return w;
}

/* ---------- batched-workload graph sizes ---------- */

/* Graph `idx` of the batched workload: kind 0 = Erdos-Renyi, 1 = R-MAT (each
 * with probability 1/2); n = floor(256 * 256^U), U uniform in [0,1), so n is
 * log-uniform in [256, 65536); mean degree uniform in [4, 64]. Draws 0..2 of
 * the graph's stream decide these; the edges use the rest. */
void gg_batch_spec(uint64_t seed, int64_t idx, int32_t* kind, int64_t* n, double* mean_deg) {
    uint64_t key = gg_stream_key(seed, (uint64_t)idx);
    *kind = (int32_t)(gg_draw(key, 0) >> 63);
    double U = u01(gg_draw(key, 1));
    int64_t nn = (int64_t)(256.0 * gg_exp2(8.0 * U));
    if (nn < 256) nn = 256;
    if (nn > 65535) nn = 65535;
    *n = nn;
    *mean_deg = 4.0 + 60.0 * u01(gg_draw(key, 2));
}

/* OpenMP threads for parallel regions started by the calling thread. */
void gg_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
