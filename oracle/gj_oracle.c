/*
 * gj_oracle.c -- plain, slow, single-threaded CPU oracle for acyclic n-way
 * equi-joins (Graphical Join, arXiv 2206.10435).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code with
 * the CUDA path and is not part of the product.
 *
 * What it computes, by definition rather than by the paper's algorithms:
 *
 *   orc_count   the join size |Q| (the partition function Z of Eq. 3) and,
 *               for every row of every relation, the number of result tuples
 *               that row takes part in.  It is a plain counting pass over
 *               ROWS (not over distinct key tuples): for a row r of relation
 *               t, up(r) = product over t's children c of the number of rows
 *               of c's subtree join that agree with r; down(r) = the number
 *               of ways to complete the rest of the tree given r.  Then
 *               |Q| = sum of up over the root's rows and every row takes
 *               part in up(r) * down(r) result tuples.  Arithmetic is exact
 *               in 128 bits and clamped to CAP = 2^64 - 1, which marks
 *               "at least 2^64 - 1"; a factor 0 beats a clamped factor
 *               (0 * CAP = 0), so dead branches never report overflow.
 *
 *   orc_join    the join result itself, as a cascade of binary hash joins
 *               over row-id tuples (relation 1 into relation 0, then
 *               relation 2 into that, ...), followed by a sort of the
 *               result into canonical order: ascending signed int32 values
 *               of the variables in the given order V, ties broken by the
 *               original row indices r_1..r_k in relation order (Def. 1
 *               sorts the result by all its columns; row ids decide among
 *               duplicate tuples of a bag).
 *
 * The join tree (parent of every relation, separator columns, V) is an
 * input; the Python side of the oracle plans it.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_CAP UINT64_MAX

typedef struct {
    int64_t n_rows;
    int32_t n_keys;
    const int32_t *const *key;   /* [n_keys] -> int32[n_rows] */
} orc_rel;

/* For relation j > 0: sep_w[j] columns; sep_cj[j][i] is the column in j,
 * sep_cp[j][i] the matching column in parent[j]. */
typedef struct {
    int32_t n_rel;
    const orc_rel *rel;
    const int32_t *parent;           /* [n_rel], parent[0] = -1, parent[j] < j */
    const int32_t *sep_w;            /* [n_rel] */
    const int32_t *const *sep_cj;    /* [n_rel] -> int32[sep_w[j]] */
    const int32_t *const *sep_cp;    /* [n_rel] -> int32[sep_w[j]] */
    int32_t n_vars;
    const int32_t *var_rel;          /* V: relation holding the variable */
    const int32_t *var_col;          /*    and its column there */
} orc_query;

/* ---------------------------------------------------------------- */
/* clamped counting arithmetic                                        */

static uint64_t clamp128(unsigned __int128 x) {
    return x >= (unsigned __int128)ORC_CAP ? ORC_CAP : (uint64_t)x;
}

static uint64_t cadd(uint64_t a, uint64_t b) {
    return clamp128((unsigned __int128)a + b);
}

static uint64_t cmul(uint64_t a, uint64_t b) {
    if (a == 0 || b == 0) return 0;
    if (a == ORC_CAP || b == ORC_CAP) return ORC_CAP;
    return clamp128((unsigned __int128)a * b);
}

/* ---------------------------------------------------------------- */
/* hash map from a tuple of w int32 values to a slot index            */

typedef struct {
    int w;
    int64_t cap;      /* power of two */
    int64_t n;
    int64_t *slot;    /* -1 empty, else entry index */
    int32_t *keys;    /* [n * w] */
    int64_t kcap;
} tmap;

static uint64_t hash_tuple(const int32_t *t, int w) {
    uint64_t h = 0x9E3779B97F4A7C15ull;
    for (int i = 0; i < w; i++) {
        h ^= (uint64_t)(uint32_t)t[i] + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
        h *= 0xBF58476D1CE4E5B9ull;
        h ^= h >> 31;
    }
    return h;
}

static int tmap_init(tmap *m, int w, int64_t expect) {
    int64_t cap = 16;
    while (cap < 2 * expect + 16) cap <<= 1;
    m->w = w; m->cap = cap; m->n = 0;
    m->slot = (int64_t *)malloc(sizeof(int64_t) * cap);
    m->kcap = expect + 16;
    m->keys = (int32_t *)malloc(sizeof(int32_t) * (size_t)(w > 0 ? w : 1) * m->kcap);
    if (!m->slot || !m->keys) return -1;
    for (int64_t i = 0; i < cap; i++) m->slot[i] = -1;
    return 0;
}

static void tmap_free(tmap *m) { free(m->slot); free(m->keys); }

/* returns the entry index of tuple t, inserting it if absent (or -1 if
 * absent and insert == 0) */
static int64_t tmap_get(tmap *m, const int32_t *t, int insert) {
    uint64_t mask = (uint64_t)m->cap - 1;
    uint64_t h = hash_tuple(t, m->w) & mask;
    for (;;) {
        int64_t e = m->slot[h];
        if (e < 0) break;
        if (memcmp(m->keys + e * m->w, t, sizeof(int32_t) * m->w) == 0) return e;
        h = (h + 1) & mask;
    }
    if (!insert) return -1;
    if (m->n == m->kcap) return -2;   /* sized by the caller; never grows */
    int64_t e = m->n++;
    memcpy(m->keys + e * m->w, t, sizeof(int32_t) * m->w);
    m->slot[h] = e;
    return e;
}

/* the separator tuple of row r of relation j, read from relation j itself
 * (from_parent = 0) or from a row r of its parent (from_parent = 1) */
static void sep_tuple(const orc_query *q, int j, int from_parent, int64_t r, int32_t *out) {
    const orc_rel *R = &q->rel[from_parent ? q->parent[j] : j];
    const int32_t *cols = from_parent ? q->sep_cp[j] : q->sep_cj[j];
    for (int i = 0; i < q->sep_w[j]; i++) out[i] = R->key[cols[i]][r];
}

/* ---------------------------------------------------------------- */
/* counting pass                                                      */

/*
 * up[j], down[j], mult[j]: caller-owned uint64[n_rows of j] (mult/down may
 * be NULL).  *total receives |Q| clamped to CAP.
 * Returns 0 if |Q| < 2^64 - 1, 1 if it is clamped (overflow), -1 on
 * allocation failure.
 */
int orc_count(const orc_query *q, uint64_t *const *up, uint64_t *const *down,
              uint64_t *const *mult, uint64_t *total) {
    int k = q->n_rel;
    int rc = 0;
    int32_t tup[64];
    /* msg[j]: map from j's separator tuple to the sum of up over j's rows */
    tmap *msg = (tmap *)calloc((size_t)k, sizeof(tmap));
    uint64_t **msgv = (uint64_t **)calloc((size_t)k, sizeof(uint64_t *));
    tmap *dmsg = (tmap *)calloc((size_t)k, sizeof(tmap));
    uint64_t **dmsgv = (uint64_t **)calloc((size_t)k, sizeof(uint64_t *));
    if (!msg || !msgv || !dmsg || !dmsgv) { rc = -1; goto done; }

    /* upward: children have larger indices than their parents */
    for (int j = k - 1; j >= 0; j--) {
        const orc_rel *R = &q->rel[j];
        for (int64_t r = 0; r < R->n_rows; r++) {
            uint64_t v = 1;
            for (int c = j + 1; c < k; c++) {
                if (q->parent[c] != j) continue;
                sep_tuple(q, c, 1, r, tup);
                int64_t e = tmap_get(&msg[c], tup, 0);
                v = cmul(v, e < 0 ? 0 : msgv[c][e]);
            }
            up[j][r] = v;
        }
        if (j == 0) break;
        if (tmap_init(&msg[j], q->sep_w[j], R->n_rows) != 0) { rc = -1; goto done; }
        msgv[j] = (uint64_t *)calloc((size_t)R->n_rows + 16, sizeof(uint64_t));
        if (!msgv[j]) { rc = -1; goto done; }
        for (int64_t r = 0; r < R->n_rows; r++) {
            sep_tuple(q, j, 0, r, tup);
            int64_t e = tmap_get(&msg[j], tup, 1);
            msgv[j][e] = cadd(msgv[j][e], up[j][r]);
        }
    }
    uint64_t t = 0;
    for (int64_t r = 0; r < q->rel[0].n_rows; r++) t = cadd(t, up[0][r]);
    *total = t;
    rc = (t == ORC_CAP) ? 1 : 0;

    if (down == NULL) goto done;
    /* downward: down(root row) = 1; for a child c of j, the ways outside
     * c's subtree given c's separator tuple s is the sum over rows r of j
     * with that tuple of down(r) times the product of j's other children */
    for (int64_t r = 0; r < q->rel[0].n_rows; r++) down[0][r] = 1;
    for (int c = 1; c < k; c++) {
        int j = q->parent[c];
        const orc_rel *P = &q->rel[j];
        if (tmap_init(&dmsg[c], q->sep_w[c], P->n_rows) != 0) { rc = -1; goto done; }
        dmsgv[c] = (uint64_t *)calloc((size_t)P->n_rows + 16, sizeof(uint64_t));
        if (!dmsgv[c]) { rc = -1; goto done; }
        for (int64_t r = 0; r < P->n_rows; r++) {
            uint64_t v = down[j][r];
            for (int c2 = j + 1; c2 < k; c2++) {
                if (q->parent[c2] != j || c2 == c) continue;
                sep_tuple(q, c2, 1, r, tup);
                int64_t e = tmap_get(&msg[c2], tup, 0);
                v = cmul(v, e < 0 ? 0 : msgv[c2][e]);
            }
            sep_tuple(q, c, 1, r, tup);
            int64_t e = tmap_get(&dmsg[c], tup, 1);
            dmsgv[c][e] = cadd(dmsgv[c][e], v);
        }
        const orc_rel *C = &q->rel[c];
        for (int64_t r = 0; r < C->n_rows; r++) {
            sep_tuple(q, c, 0, r, tup);
            int64_t e = tmap_get(&dmsg[c], tup, 0);
            down[c][r] = e < 0 ? 0 : dmsgv[c][e];
        }
    }
    if (mult != NULL)
        for (int j = 0; j < k; j++)
            for (int64_t r = 0; r < q->rel[j].n_rows; r++)
                mult[j][r] = cmul(up[j][r], down[j][r]);

done:
    for (int j = 0; j < k; j++) {
        if (msg && msg[j].slot) tmap_free(&msg[j]);
        if (msgv) free(msgv[j]);
        if (dmsg && dmsg[j].slot) tmap_free(&dmsg[j]);
        if (dmsgv) free(dmsgv[j]);
    }
    free(msg); free(msgv); free(dmsg); free(dmsgv);
    return rc;
}

/* ---------------------------------------------------------------- */
/* cascade of binary hash joins + canonical sort                      */

static const orc_query *g_q;      /* comparator context (single thread) */
static const int32_t *g_tuples;

static int cmp_canonical(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    int k = g_q->n_rel;
    const int32_t *ta = g_tuples + a * k, *tb = g_tuples + b * k;
    for (int v = 0; v < g_q->n_vars; v++) {
        int rel = g_q->var_rel[v], col = g_q->var_col[v];
        int32_t x = g_q->rel[rel].key[col][ta[rel]];
        int32_t y = g_q->rel[rel].key[col][tb[rel]];
        if (x != y) return x < y ? -1 : 1;
    }
    for (int j = 0; j < k; j++)
        if (ta[j] != tb[j]) return ta[j] < tb[j] ? -1 : 1;
    return 0;
}

/*
 * Materialises the join as row-id tuples.  out: int32[cap * n_rel], tuple i
 * at out[i*n_rel .. ], canonical order.  inter[j] (j = 0..n_rel-1) receives
 * the size of the intermediate result after joining relations 0..j.
 * Returns |Q|, -2 if an intermediate result would exceed max_tuples, -1 on
 * allocation failure.
 */
int64_t orc_join(const orc_query *q, int32_t *out, int64_t cap, int64_t max_tuples,
                 int64_t *inter) {
    int k = q->n_rel;
    int32_t tup[64];
    int64_t n = q->rel[0].n_rows;
    if (n > max_tuples) return -2;
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1) * k);
    if (!cur) return -1;
    for (int64_t r = 0; r < n; r++) cur[r * k] = (int32_t)r;
    inter[0] = n;
    for (int j = 1; j < k; j++) {
        const orc_rel *R = &q->rel[j];
        int p = q->parent[j];
        /* build side: relation j hashed on its separator tuple, rows chained
         * in increasing order */
        tmap m;
        if (tmap_init(&m, q->sep_w[j], R->n_rows) != 0) { free(cur); return -1; }
        int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)(R->n_rows + 1));
        int64_t *tail = (int64_t *)malloc(sizeof(int64_t) * (size_t)(R->n_rows + 1));
        int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(R->n_rows + 1));
        if (!head || !tail || !next) { free(cur); return -1; }
        for (int64_t r = 0; r < R->n_rows; r++) {
            sep_tuple(q, j, 0, r, tup);
            tmap_get(&m, tup, 1);
            next[r] = -1;
        }
        for (int64_t e = 0; e < m.n; e++) head[e] = tail[e] = -1;
        for (int64_t r = 0; r < R->n_rows; r++) {
            sep_tuple(q, j, 0, r, tup);
            int64_t e = tmap_get(&m, tup, 0);
            if (head[e] < 0) head[e] = r; else next[tail[e]] = r;
            tail[e] = r;
        }
        /* probe side: current tuples, via their parent row */
        int64_t cnt = 0;
        for (int64_t i = 0; i < n; i++) {
            sep_tuple(q, j, 1, cur[i * k + p], tup);
            int64_t e = tmap_get(&m, tup, 0);
            if (e < 0) continue;
            for (int64_t r = head[e]; r >= 0; r = next[r]) cnt++;
        }
        if (cnt > max_tuples) {
            tmap_free(&m); free(head); free(tail); free(next); free(cur);
            return -2;
        }
        int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1) * k);
        if (!nxt) { tmap_free(&m); free(head); free(tail); free(next); free(cur); return -1; }
        int64_t o = 0;
        for (int64_t i = 0; i < n; i++) {
            sep_tuple(q, j, 1, cur[i * k + p], tup);
            int64_t e = tmap_get(&m, tup, 0);
            if (e < 0) continue;
            for (int64_t r = head[e]; r >= 0; r = next[r]) {
                memcpy(nxt + o * k, cur + i * k, sizeof(int32_t) * j);
                nxt[o * k + j] = (int32_t)r;
                o++;
            }
        }
        tmap_free(&m); free(head); free(tail); free(next); free(cur);
        cur = nxt;
        n = cnt;
        inter[j] = n;
    }
    if (n > cap) { free(cur); return -2; }
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!idx) { free(cur); return -1; }
    for (int64_t i = 0; i < n; i++) idx[i] = i;
    g_q = q; g_tuples = cur;
    qsort(idx, (size_t)n, sizeof(int64_t), cmp_canonical);
    for (int64_t i = 0; i < n; i++) memcpy(out + i * k, cur + idx[i] * k, sizeof(int32_t) * k);
    free(idx); free(cur);
    return n;
}
