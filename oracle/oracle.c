/*
 * oracle.c -- the CPU oracle for exact triangle counting.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct
 * reference that the CUDA path is checked against. Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline / reference arm may
 * load it. It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (TRUST, Sec. 1 and Sec. 2.2): the number of triangles
 * (three-vertex cliques) of a simple undirected graph,
 *     T(G) = #{ {a,b,c} : ab, bc, ca are edges }.
 * Three routes to that number live here:
 *   oracle_brute       -- the definition itself, a triple loop over a dense
 *                         adjacency matrix (tiny graphs only);
 *   oracle_orient      -- rank-by-degree orientation (Sec. 2.2): every
 *                         undirected edge {u,v} is kept once, directed from the
 *                         lower to the higher (degree, id) pair;
 *   oracle_count_dag   -- node iterator with merge-path intersection (Sec. 2.2,
 *                         "merge-path based intersection"): for every u and
 *                         every v in N+(u), |N+(u) ∩ N+(v)| by a two-pointer
 *                         walk over the sorted lists, summed in uint64. Each
 *                         triangle a < b < c (in the orientation order) is
 *                         counted exactly once, at u = a, v = b, w = c.
 * The input is the symmetric CSR of Sec. 2.1 (begin positions + adjacency
 * list); row_ptr is int64 here, col int32, rows in any order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ brute */

/* T(G) from the definition: for every a < b < c, test the three edges in a
 * dense 0/1 adjacency matrix. n <= 4096. Returns UINT64_MAX if n is too big
 * or memory runs out. */
uint64_t oracle_brute(int64_t n, const int64_t* row_ptr, const int32_t* col) {
    if (n > 4096) return UINT64_MAX;
    if (n < 3) return 0;
    unsigned char* adj = (unsigned char*)calloc((size_t)(n * n), 1);
    if (!adj) return UINT64_MAX;
    for (int64_t u = 0; u < n; u++)
        for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; k++) {
            int64_t v = col[k];
            if (v != u) { adj[u * n + v] = 1; adj[v * n + u] = 1; }
        }
    uint64_t t = 0;
    for (int64_t a = 0; a < n; a++)
        for (int64_t b = a + 1; b < n; b++) {
            if (!adj[a * n + b]) continue;
            for (int64_t c = b + 1; c < n; c++)
                if (adj[b * n + c] && adj[a * n + c]) t++;
        }
    free(adj);
    return t;
}

/* -------------------------------------------------------------- orientation */

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Strict total order "u precedes v" used for orientation. With key == NULL it
 * is rank-by-degree (Sec. 2.2): compare undirected degrees, ties broken by
 * vertex id. With a key array it is the order of key[] (keys must be distinct),
 * which lets tests check that the count does not depend on the order. */
static inline int precedes(int64_t u, int64_t v, const int64_t* row_ptr, const int64_t* key) {
    if (key) return key[u] < key[v];
    int64_t du = row_ptr[u + 1] - row_ptr[u], dv = row_ptr[v + 1] - row_ptr[v];
    if (du != dv) return du < dv;
    return u < v;
}

static int64_t orient_impl(int64_t n, const int64_t* row_ptr, const int32_t* col, const int64_t* key,
                           int64_t* dag_ptr, int32_t* dag_col) {
    /* pass 1: out-degree of every vertex */
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t u = 0; u < n; u++) {
        int64_t c = 0;
        for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; k++)
            if (precedes(u, col[k], row_ptr, key)) c++;
        dag_ptr[u + 1] = c;
    }
    dag_ptr[0] = 0;
    for (int64_t u = 0; u < n; u++) dag_ptr[u + 1] += dag_ptr[u];
    /* pass 2: write and sort N+(u) */
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t u = 0; u < n; u++) {
        int64_t w = dag_ptr[u];
        for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; k++)
            if (precedes(u, col[k], row_ptr, key)) dag_col[w++] = col[k];
        qsort(dag_col + dag_ptr[u], (size_t)(dag_ptr[u + 1] - dag_ptr[u]), sizeof(int32_t), cmp_i32);
    }
    return dag_ptr[n];
}

/* Rank-by-degree orientation. dag_ptr: n+1 entries; dag_col: room for
 * row_ptr[n]/2 entries (every undirected edge is kept once). Rows of the
 * result are sorted ascending. Returns the number of DAG edges m. */
int64_t oracle_orient(int64_t n, const int64_t* row_ptr, const int32_t* col, int64_t* dag_ptr,
                      int32_t* dag_col) {
    return orient_impl(n, row_ptr, col, NULL, dag_ptr, dag_col);
}

/* Orientation by an arbitrary strict order given as distinct keys. */
int64_t oracle_orient_by_key(int64_t n, const int64_t* row_ptr, const int32_t* col, const int64_t* key,
                             int64_t* dag_ptr, int32_t* dag_col) {
    return orient_impl(n, row_ptr, col, key, dag_ptr, dag_col);
}

/* ---------------------------------------------------------------- counting */

/* |A ∩ B| of two ascending lists by the two-pointer (merge-path) walk. */
static uint64_t merge_count(const int32_t* a, int64_t na, const int32_t* b, int64_t nb) {
    uint64_t c = 0;
    int64_t i = 0, j = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) i++;
        else if (a[i] > b[j]) j++;
        else { c++; i++; j++; }
    }
    return c;
}

/* Triangles whose lowest vertex in the orientation order is u:
 * sum over v in N+(u) of |N+(u) ∩ N+(v)|. Rows must be sorted. */
static uint64_t apex_count(int64_t u, const int64_t* dag_ptr, const int32_t* dag_col) {
    const int32_t* nu = dag_col + dag_ptr[u];
    int64_t du = dag_ptr[u + 1] - dag_ptr[u];
    uint64_t t = 0;
    for (int64_t k = 0; k < du; k++) {
        int64_t v = nu[k];
        t += merge_count(nu, du, dag_col + dag_ptr[v], dag_ptr[v + 1] - dag_ptr[v]);
    }
    return t;
}

static void set_threads(int threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
}

/* Node iterator over a DAG with sorted rows: T = sum_u apex(u). per_vertex
 * (n entries, may be NULL) receives apex(u). threads <= 0: library default. */
uint64_t oracle_count_dag(int64_t n, const int64_t* dag_ptr, const int32_t* dag_col, uint64_t* per_vertex,
                          int threads) {
    set_threads(threads);
    uint64_t total = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : total)
    for (int64_t u = 0; u < n; u++) {
        uint64_t t = apex_count(u, dag_ptr, dag_col);
        if (per_vertex) per_vertex[u] = t;
        total += t;
    }
    return total;
}

/* apex(u) for the k vertices us[0..k). */
void oracle_count_dag_at(int64_t n, const int64_t* dag_ptr, const int32_t* dag_col, int64_t k,
                         const int64_t* us, uint64_t* out, int threads) {
    (void)n;
    set_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < k; i++) out[i] = apex_count(us[i], dag_ptr, dag_col);
}

/* orient + count in one call. Returns UINT64_MAX on allocation failure. */
uint64_t oracle_count(int64_t n, const int64_t* row_ptr, const int32_t* col, int threads) {
    set_threads(threads);
    int64_t* dag_ptr = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    int32_t* dag_col = (int32_t*)malloc((size_t)(row_ptr[n] / 2 + 1) * sizeof(int32_t));
    if (!dag_ptr || !dag_col) { free(dag_ptr); free(dag_col); return UINT64_MAX; }
    orient_impl(n, row_ptr, col, NULL, dag_ptr, dag_col);
    uint64_t t = oracle_count_dag(n, dag_ptr, dag_col, NULL, threads);
    free(dag_ptr);
    free(dag_col);
    return t;
}

/* ------------------------------------------------------------- reordering */

/* The two vertex reorderings of Sec. 4.1, which change vertex ids (and so the
 * buckets ids hash to) but never the count. Both run on the oriented graph
 * N+ (rows sorted ascending, as oracle_orient leaves them):
 *   kind 1, by in-degree: sort the vertices by in-degree in N+ (the number of
 *     lists N+(u) that contain v), largest first, ties by smaller old id, and
 *     number them 0, 1, 2, ... in that order;
 *   kind 2, neighbours of the largest collective out-degree first: sort the
 *     vertices u by sum_{v in N+(u)} d+(v), largest first, ties by smaller old
 *     id; walk them in that order and give every v of N+(u), taken in
 *     ascending old id, the next new id unless it has one; vertices that got
 *     none (they are in no list) follow in ascending old id.
 * new_id[old] receives the new id. Returns 0, or -1 on a bad kind or when
 * memory runs out. */
typedef struct {
    uint64_t key;
    int64_t id;
} key_id;

static int cmp_key_desc_id_asc(const void* a, const void* b) {
    const key_id* x = (const key_id*)a;
    const key_id* y = (const key_id*)b;
    if (x->key != y->key) return x->key > y->key ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

int oracle_reorder(int64_t n, const int64_t* dag_ptr, const int32_t* dag_col, int kind, int32_t* new_id) {
    if (kind != 1 && kind != 2) return -1;
    key_id* order = (key_id*)malloc((size_t)(n > 0 ? n : 1) * sizeof(key_id));
    if (!order) return -1;
    for (int64_t u = 0; u < n; u++) {
        order[u].id = u;
        order[u].key = 0;
    }
    if (kind == 1) {
        for (int64_t e = 0; e < dag_ptr[n]; e++) order[dag_col[e]].key++;
    } else {
        for (int64_t u = 0; u < n; u++)
            for (int64_t e = dag_ptr[u]; e < dag_ptr[u + 1]; e++) {
                int64_t v = dag_col[e];
                order[u].key += (uint64_t)(dag_ptr[v + 1] - dag_ptr[v]);
            }
    }
    qsort(order, (size_t)n, sizeof(key_id), cmp_key_desc_id_asc);
    if (kind == 1) {
        for (int64_t r = 0; r < n; r++) new_id[order[r].id] = (int32_t)r;
        free(order);
        return 0;
    }
    int64_t max_d = 0;
    for (int64_t u = 0; u < n; u++)
        if (dag_ptr[u + 1] - dag_ptr[u] > max_d) max_d = dag_ptr[u + 1] - dag_ptr[u];
    int32_t* list = (int32_t*)malloc((size_t)(max_d > 0 ? max_d : 1) * sizeof(int32_t));
    if (!list) {
        free(order);
        return -1;
    }
    for (int64_t v = 0; v < n; v++) new_id[v] = -1;
    int64_t next = 0;
    for (int64_t r = 0; r < n; r++) {
        int64_t u = order[r].id, d = dag_ptr[u + 1] - dag_ptr[u];
        memcpy(list, dag_col + dag_ptr[u], (size_t)d * sizeof(int32_t));
        qsort(list, (size_t)d, sizeof(int32_t), cmp_i32);
        for (int64_t k = 0; k < d; k++)
            if (new_id[list[k]] < 0) new_id[list[k]] = (int32_t)next++;
    }
    for (int64_t v = 0; v < n; v++)
        if (new_id[v] < 0) new_id[v] = (int32_t)next++;
    free(list);
    free(order);
    return 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
