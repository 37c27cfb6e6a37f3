/*
 * gj.h -- C ABI of the GB300 Graphical Join library (libgj.so).
 *
 * Graphical Join (Shanghooshabad & Triantafillou, arXiv 2206.10435) computes
 * an acyclic n-way equi-join in three steps, all of them CUDA kernels here:
 *
 *   1. factor construction (Section 3.2): every relation is scanned once and
 *      grouped by its join-key tuple, giving the exact frequency table
 *      ("potential") of the relation;
 *   2. summarisation (Section 3.3, Algorithm 2; Section 3.5, Algorithms 3-4):
 *      a sum-product pass over the join tree in the counting semiring,
 *      leaves to root and back, giving the join size |Q| (the partition
 *      function Z of Eq. 3), per key-tuple result multiplicities and the
 *      offsets that place every distinct key path in the sorted result;
 *   3. desummarisation (Section 3.6): any window of rows of the sorted join
 *      result is expanded from that summary into caller-owned columns.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Pointers named "dev" or documented as device pointers must be CUDA
 *   device memory of the context's device (torch tensors qualify); all other
 *   pointers are host memory.
 * - All work is enqueued on the context's stream.  Calls that return a host
 *   value computed on the device (gj_summarize, gj_query_sizes, gj_level,
 *   gj_desummarize's *n_out) synchronise that stream before returning.
 * - Errors are returned, never raised: no call aborts the process and no
 *   kernel traps.  Device-side waits are bounded and report GJ_ERR_TIMEOUT.
 * - Counts are exact unsigned 64-bit integers.  UINT64_MAX is reserved as
 *   the saturation marker: a join whose size is 2^64 - 1 or more reports
 *   GJ_ERR_OVERFLOW.  A dead branch (a zero count) never overflows.
 * - Limits: a relation holds at most 2^31 - 1 rows and at most 8 key
 *   columns; a query joins at most 16 relations.  Key values are int32 and
 *   ordered as signed integers.
 */
#ifndef GJ_H
#define GJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GJ_OK = 0,
    GJ_ERR_INVALID = 1,      /* bad argument, unknown id, size beyond a limit */
    GJ_ERR_NOT_ACYCLIC = 2,  /* relation order does not give a join tree */
    GJ_ERR_OOM = 3,          /* device allocation failed */
    GJ_ERR_OVERFLOW = 4,     /* |Q| >= 2^64 - 1 */
    GJ_ERR_CUDA = 5,         /* a CUDA runtime call failed */
    GJ_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
    GJ_ERR_STATE = 7,        /* call out of order (e.g. desummarise before summarise) */
    GJ_ERR_CAPACITY = 8      /* caller's output buffer too small; *n_out holds the need */
} gj_status;

typedef struct gj_ctx gj_ctx;
typedef struct gj_query gj_query;

/* Relation columns live on the device unless GJ_REL_HOST is set. */
#define GJ_REL_BORROW 0u     /* keep the caller's device pointers; caller keeps them alive */
#define GJ_REL_COPY 1u       /* copy the columns into library-owned device memory */
#define GJ_REL_HOST 2u       /* columns are host pointers; implies a copy (H2D) */

/*
 * One relation (a table of the join, Section 1.1).  Key columns are the join
 * attributes: two relations join on every attribute id they share.  Payload
 * columns are the non-join attributes, conditionally independent of each
 * other given the join attributes (Section 3.2), and are carried by row id.
 */
typedef struct {
    int64_t n_rows;
    int32_t n_keys;                    /* 1..8 */
    const int32_t *key_attr;           /* [n_keys] attribute id of every key column */
    const int32_t *const *key_cols;    /* [n_keys] -> int32[n_rows] */
    int32_t n_payloads;                /* 0..8 */
    const int32_t *payload_width;      /* [n_payloads] bytes per value: 4 or 8 */
    const void *const *payload_cols;   /* [n_payloads] -> width * n_rows bytes */
    uint32_t flags;                    /* GJ_REL_* */
} gj_relation_desc;

/* Result-shape description of a query (filled by gj_query_sizes). */
typedef struct {
    int32_t n_rel;
    int32_t n_vars;                    /* |V|: key columns of the result */
    int32_t var_attr[64];              /* attribute id of result key column i */
    int32_t n_cols;                    /* n_vars + all payload columns */
    int32_t col_width[64];             /* bytes per value of result column i */
    int32_t parent[16];                /* join tree: parent relation, -1 for the root */
    int64_t n_groups[16];              /* distinct key tuples per relation */
} gj_query_sizes_t;

/* Counters of gj_profile. */
typedef struct {
    uint64_t launches;       /* kernels the context launched since the last read */
    uint64_t emit_launches;  /* launches of the desummarise emit kernel while profiling */
    double emit_ms;          /* their summed device time, from CUDA events on the stream */
    uint64_t emit_rows;      /* result rows they wrote */
    uint64_t emit_bytes;     /* bytes of result columns they wrote */
    double expand_ms;        /* time from the start to the end of the window expansions
                                (Algorithm 4 restricted to each window), CUDA events */
} gj_profile_t;

/* Library version and status text. */
const char *gj_status_str(gj_status s);
int32_t gj_version(void);
/* The last CUDA failure seen by this thread: error name, text, source line. */
const char *gj_last_error(void);

/*
 * Creates a context on CUDA device `device` that enqueues its work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * The context owns relations, factors and queries; gj_destroy frees them.
 */
gj_status gj_create(gj_ctx **out, int32_t device, void *cuda_stream);
void gj_destroy(gj_ctx *ctx);
gj_status gj_set_stream(gj_ctx *ctx, void *cuda_stream);

/*
 * Tuning options of a context (no counterpart in the paper).
 * GJ_OPT_EMIT_ROWS_PER_THREAD: result rows each thread of the desummarise
 * emit kernel writes, 2, 4 or 8 (default 4): fewer rows per thread means fewer
 * registers and more threads in flight, more rows means fewer block
 * lookups per row.  Takes effect for queries created afterwards.
 * GJ_OPT_TRIANGLE_INTERSECT: how the cyclic 3-way join finds the group
 * triples of its maxclique potential (Section 3.2.1): 0 (default) chooses
 * by the key ranges and segment lengths, 1 sorted-list intersection,
 * 2 bitmaps over C's value range (rows per value of B in S and of A in T;
 * used only while they take at most 512 MiB, else lists).  The triples and
 * their order are the same either way.  Takes effect at the next
 * gj_summarize.
 * GJ_OPT_DOWN_COMBINE: how the downward pass (Algorithm 2's messages back
 * down the tree) adds the contributions of a relation's groups to a
 * child's down message: 0 (default) combines them per thread block in
 * shared memory first where the links to that child are not in key order
 * (so skewed keys do not serialise on one address), 1 never, 2 for every
 * child.  The sums are exact integers: the summary is the same either way.
 * Takes effect at the next gj_summarize.
 * GJ_OPT_SLOT_ARENA: bytes of the bump arena each slot of a server created
 * afterwards takes its requests' device memory from (default 512 MiB, 0 =
 * none: every allocation goes to the slot's memory pool; at most 2^40).  A
 * request that needs more continues in the pool; results are the same.
 * Unknown options and values outside these ranges return GJ_ERR_INVALID
 * and change nothing; a NULL ctx returns GJ_ERR_INVALID.
 */
#define GJ_OPT_EMIT_ROWS_PER_THREAD 1
#define GJ_OPT_TRIANGLE_INTERSECT 2
#define GJ_OPT_DOWN_COMBINE 6
#define GJ_OPT_SLOT_ARENA 7
gj_status gj_set_option(gj_ctx *ctx, int32_t option, int64_t value);

/*
 * Failure injection, for tests of the error paths (no counterpart in the
 * paper).  None of them can hang or fault the device.
 * GJ_OPT_SPIN_LIMIT: polls after which the bounded wait of the factor
 * build's group scan (a tile waiting on its predecessors' counts) gives up,
 * 1 .. 2^22; 0 restores the default (2^22).
 * GJ_OPT_TEST_STALL: 1 makes the first tile of that scan never publish its
 * count, so every other tile's wait runs out: the factor build reports
 * GJ_ERR_TIMEOUT (its results are discarded, every array stays in
 * bounds), and the context stays usable; 0 turns it off.
 * GJ_OPT_FAIL_ALLOC_AT: N > 0 makes the N-th device allocation of the
 * context from now on fail as if the device were out of memory (the call
 * returns GJ_ERR_OOM and frees what it had allocated); 0 turns it off.
 */
#define GJ_OPT_SPIN_LIMIT 3
#define GJ_OPT_TEST_STALL 4
#define GJ_OPT_FAIL_ALLOC_AT 5

/*
 * Device memory the context's pool has handed out and not taken back
 * (bytes; waits for the context's stream first), and the device
 * allocations the context has made since GJ_OPT_FAIL_ALLOC_AT was last set
 * (either pointer may be NULL).  No counterpart in the paper.
 */
gj_status gj_pool_usage(gj_ctx *ctx, uint64_t *used_bytes, int64_t *allocations);

/*
 * Profiling (no counterpart in the paper, which reports wall-clock times
 * only).  With out != NULL: synchronises the stream, writes the counters
 * accumulated since the previous read and resets them.  Then turns device
 * timing of the emit kernel on (enable != 0) or off.
 */
gj_status gj_profile(gj_ctx *ctx, int32_t enable, gj_profile_t *out);

/*
 * Registers a relation (Section 1.1: the tables T_1..T_n to be joined).
 * Column pointers are device pointers (GJ_REL_BORROW, GJ_REL_COPY) or host
 * pointers (GJ_REL_HOST).  Borrowed columns must outlive the relation.
 * Returns its id in *rel_id.
 */
gj_status gj_load_relation(gj_ctx *ctx, const gj_relation_desc *desc, int32_t *rel_id);
gj_status gj_release_relation(gj_ctx *ctx, int32_t rel_id);

/*
 * Factor construction (Section 3.2, "quantitative learning"): groups the
 * relation's rows by their key tuple, ordered by the columns in `col_order`
 * (a permutation of 0..n_keys-1, most significant first; NULL = declared
 * order), rows of a group in increasing row id.  The result is the exact
 * frequency table of the relation: distinct key tuples with their counts.
 * Idempotent and cached per column order; factors may be built ahead of any
 * query and reused by many (Section 3.2, last paragraph; Section 4.1).
 */
gj_status gj_build_factors(gj_ctx *ctx, int32_t rel_id, const int32_t *col_order);

/*
 * Exports a built factor: *n_groups, and, for non-NULL device outputs,
 * perm (uint32[n_rows], row ids in group order), gstart (uint32[n_groups+1],
 * first position of every group in perm) and gkey (int32[n_keys*n_groups],
 * key column c of group g at gkey[c*n_groups + g]).  Call once with NULL
 * outputs to learn n_groups.
 */
gj_status gj_factor_export(gj_ctx *ctx, int32_t rel_id, const int32_t *col_order,
                           int64_t *n_groups, uint32_t *perm_dev, uint32_t *gstart_dev,
                           int32_t *gkey_dev);

/*
 * Plans a query over relations rel_ids[0..n_rel-1] (rel_ids[0] is the root).
 * Relation j > 0 hangs under the first earlier relation that holds every
 * attribute j shares with relations 0..j-1; if j shares nothing the query
 * is rejected (GJ_ERR_INVALID); if no earlier relation holds them all the
 * order gives no join tree and the query is cyclic (below).  The result's key columns V are a preorder
 * walk of that tree, every relation adding the attributes its parent lacks
 * in declared column order; payload columns follow, relation by relation.
 * Rows of the result are ordered by V (signed int32, ascending), ties broken
 * by the original row ids r_1..r_k (Def. 1 sorts the result by all columns).
 * Builds any factor it needs.
 *
 * Cyclic queries (Sections 3.2.1, 3.4; 2 to 8 relations, every relation
 * after the first sharing an attribute with those before it) are answered
 * over a junction tree: the summary is the joint potential of its
 * maxcliques (Algorithm 1: the factors joined, frequencies multiplied), as
 * blocks of one group per relation.  The 3-cycle R0(A,B) R1(B,C) R2(C,A)
 * (two key columns each, any column order) uses the maxclique {A,B,C};
 * other shapes use two maxcliques (relations 0-1 and the rest, joined on
 * their common attributes) where every relation of the second clique after
 * its first shares an attribute with the ones before it and the second
 * clique's attributes pack into 64 bits, else one maxclique holding every
 * attribute.  V is the attributes in order of first
 * appearance (relation 0's columns in declared order, then each relation's
 * new attributes in declared order); rows are ordered as above.  Queries
 * whose intermediate blocks would exceed 2^31 return GJ_ERR_OOM.
 * gj_summarize and gj_desummarize work as for a tree; gj_level,
 * gj_summary_groups, gj_summary_save and the row-sharded counting calls
 * return GJ_ERR_INVALID for them.
 */
gj_status gj_query_create(gj_ctx *ctx, const int32_t *rel_ids, int32_t n_rel, gj_query **out);

/*
 * Early projection (Section 3.7): gj_query_create for a result without the
 * attributes drop_attrs[0..n_drop-1].  Those variables are deleted from the
 * model before the summary is built: V omits them, gj_desummarize writes no
 * column for them and the rows are ordered by the remaining variables of V,
 * ties broken by the row ids r_1..r_k.  The result keeps bag semantics: it
 * holds the same |Q| row-id tuples as the full join, only without the
 * dropped columns and in that order.
 * Supported: attributes that occur in exactly one relation of the query.
 * That relation's factor groups its rows by its remaining key columns, so
 * it has fewer groups and the summary shrinks.  A join attribute (shared by
 * two relations; deleting it needs the potential join of Algorithm 1), an
 * attribute no relation holds, or a root left without key columns gives
 * GJ_ERR_INVALID.
 */
gj_status gj_query_create_projected(gj_ctx *ctx, const int32_t *rel_ids, int32_t n_rel,
                                    const int32_t *drop_attrs, int32_t n_drop, gj_query **out);
void gj_query_destroy(gj_query *q);
gj_status gj_query_sizes(gj_query *q, gj_query_sizes_t *out);

/*
 * Runs this query's later work (summarise, levels, desummarise, destroy) on
 * its own stream with its own readback buffer and error word, sharing the
 * context's relations, factors and memory pool.  Different queries may then
 * be driven from different host threads at the same time and their kernels
 * overlap on the device.  Loading, releasing, factor building and query
 * creation are serialised by a lock inside the context.
 */
gj_status gj_query_set_stream(gj_query *q, void *cuda_stream);

/*
 * Summarisation: the upward sum-product pass of Algorithm 2 over the join
 * tree in the counting semiring (Eqs. 4-10: product of a relation's
 * frequencies with its children's messages, summed out over the separator),
 * the root marginal whose sum is the join size (Section 3.3), and the
 * downward pass that gives every distinct key tuple of every relation its
 * result multiplicity and every key path its offset in the sorted result
 * (the bucket products of Algorithm 4).  Writes |Q| to *total (UINT64_MAX
 * when GJ_ERR_OVERFLOW).  Synchronises the stream.
 */
gj_status gj_summarize(gj_query *q, uint64_t *total);

/*
 * Per-group summary of relation position `rel` (0..n_rel-1) of the query,
 * into device arrays of n_groups entries each (any may be NULL):
 *   w:     result rows per (key tuple, fixed ancestors) = count x product of
 *          the children's messages (the bucket * fac of Section 3.3)
 *   mult:  number of result tuples that use the key tuple (its marginal
 *          over the join result, Section 1.2 "Why PGMs")
 *   off:   for the root, the first result row of the key tuple; for other
 *          relations, the exclusive prefix of w within its separator segment
 * Group order is the factor's (separator columns first).
 */
gj_status gj_summary_groups(gj_query *q, int32_t rel, uint64_t *w_dev, uint64_t *mult_dev,
                            uint64_t *off_dev);

/*
 * GFJS column `level` (0..n_vars-1; Def. 1, Figure 2): the runs of the
 * sorted result over distinct prefixes (v_0..v_level), one run per prefix
 * (Algorithm 4 emits one entry per prefix), restricted to runs that START
 * in result rows [row0, row0 + n_rows).  Writes value (int32), freq and
 * offset (uint64) of each run into device arrays of capacity `cap`; *n_out
 * receives the number of runs (GJ_ERR_CAPACITY if above cap).  Window rules
 * as for gj_desummarize; a level outside 0..n_vars-1 is GJ_ERR_INVALID.
 */
gj_status gj_level(gj_query *q, int32_t level, uint64_t row0, uint64_t n_rows,
                   int32_t *value_dev, uint64_t *freq_dev, uint64_t *offset_dev,
                   uint64_t cap, uint64_t *n_out);

/*
 * Desummarisation (Section 3.6): writes result rows [row0, row0 + n_rows)
 * (clipped to |Q|) into caller-owned columns out_cols[0..n_cols-1]
 * (layout from gj_query_sizes: the V key columns as int32, then payloads).
 * If rowid_cols is non-NULL, rowid_cols[j] (uint32[n_rows], may be NULL per
 * relation) receives the row id r_j of every result row.
 * Every column is either device memory of the context's device (or managed
 * memory) or pinned host memory the device can address (cudaHostAlloc,
 * cudaHostRegister; torch pin_memory()): the emit kernel then stores the
 * rows straight into host memory over the host link, without a device
 * staging buffer or a copy.  Pageable host memory is rejected
 * (GJ_ERR_INVALID).  *n_out receives the number of rows written; the rows
 * are in place once the context's stream reaches this point (the call
 * synchronises it).  Requires gj_summarize (else GJ_ERR_STATE; after an
 * overflow, GJ_ERR_OVERFLOW).  A window of no rows, or starting at or past
 * |Q|, writes nothing (*n_out = 0); one that reaches past |Q| is clipped
 * (n_rows may be up to UINT64_MAX); a clipped window of more than
 * 2^31 - 1 rows is GJ_ERR_INVALID, refused before anything is written.
 */
gj_status gj_desummarize(gj_query *q, uint64_t row0, uint64_t n_rows,
                         void *const *out_cols, uint32_t *const *rowid_cols, uint64_t *n_out);

/*
 * Batched summaries: many independent queries at once.  The paper has one
 * query at a time; the batch runs the same upward pass (Algorithm 2, the
 * root marginal summing to |Q|, Section 3.3) for every query together, so
 * its cost is a fixed sequence of about 30 kernels instead of tens of
 * launches and several synchronisations per query.
 *
 * gj_batch_create plans queries q = 0..n_queries-1, query q being the
 * relations rel_ids[query_off[q] .. query_off[q+1]) (root first, same tree
 * rules as gj_query_create).  The batched kernels take queries whose
 * relations have one or two key columns and share one attribute with their
 * parent (at most 2^32 - 1 rows in all); any other acyclic query (three or
 * more key columns, separators of several attributes) is planned as a single
 * query and summarised by gj_batch_run after the batched kernels, writing
 * its slot of the same arrays.  Planning reads the key ranges (one
 * synchronisation) and allocates the workspace; relations must stay loaded
 * and unchanged while the batch lives.
 *
 * gj_batch_run enqueues the whole summary on the context's stream without
 * any synchronisation and writes |Q| (UINT64_MAX on overflow) to
 * totals_dev[q] and GJ_OK / GJ_ERR_OVERFLOW to status_dev[q] (may be NULL).
 * With use_graph != 0 the sequence is captured into a CUDA graph on the
 * first call (and again when the outputs or parameters change) and each
 * call is one graph launch.  Queries planned as single queries run outside
 * the graph, on the same stream after it, and the call then waits for the
 * stream.
 */
typedef struct gj_batch gj_batch;
#define GJ_BATCH_GRID_MULT 1   /* persistent grids = SMs x this (1..64, default 4) */
gj_status gj_batch_create(gj_ctx *ctx, const int32_t *rel_ids, const int32_t *query_off,
                          int32_t n_queries, gj_batch **out);
gj_status gj_batch_set(gj_batch *batch, int32_t param, int64_t value);
gj_status gj_batch_info(gj_batch *batch, int64_t *n_rows, int32_t *n_relations, int32_t *levels,
                        int32_t *key_bits);
gj_status gj_batch_run(gj_batch *batch, int32_t use_graph, uint64_t *totals_dev,
                       int32_t *status_dev);
void gj_batch_destroy(gj_batch *batch);

/*
 * Compute-and-reuse (Sections 3.6 and 4, Tables 3-4): instead of storing the
 * join result, store its summary and desummarise it later.
 * gj_summary_save writes everything desummarisation needs -- per relation
 * the factor (row order, group starts and keys, payloads in group order)
 * and the summary arrays, plus the join tree and output layout -- to the
 * file `path` and reports its size in *bytes.  Requires gj_summarize.
 * gj_summary_load reads such a file into a new query on `ctx` that owns its
 * device copies and needs none of the original relations: gj_desummarize,
 * gj_level, gj_summary_groups and gj_query_sizes work on it as on the
 * original, and gj_summarize returns the stored |Q|.  A file that is not a
 * complete summary gives GJ_ERR_INVALID.
 */
gj_status gj_summary_save(gj_query *q, const char *path, uint64_t *bytes);
gj_status gj_summary_load(gj_ctx *ctx, const char *path, gj_query **out);

/*
 * Native serving runtime (Section 4.1's pre-built potentials kept resident,
 * queries answered as they arrive).  gj_server_run replays a trace of
 * n_requests queries -- request i is the relations rel_ids[query_off[i] ..
 * query_off[i+1]), arriving arrival_offsets[i] seconds after the start --
 * and returns when all are answered.  A dispatcher thread releases and
 * plans requests at their arrival times; admission is FIFO while the
 * device memory the context's pool has handed out plus the next request's
 * estimate stays under hbm_budget (a request that cannot fit with nothing
 * in flight is refused with GJ_ERR_OOM); n_slots slot threads, each with its
 * own stream, summarise a request and stream its result rows in chunks of
 * chunk_rows (up to max_rows rows per request, 0 = the whole result)
 * through the slot's buffers, so concurrent requests overlap on the device.
 * results[i] receives |Q|, the status, the rows streamed and an
 * order-independent, position-dependent 64-bit hash of all of them, and
 * arrival / admission / summary / first-chunk / last-chunk times (steady
 * clock, s).  Relations must be loaded, and their factors should be built,
 * beforehand.
 */
typedef struct gj_server gj_server;
typedef struct {
    uint64_t total;
    int32_t status;
    int32_t slot;
    uint64_t rows;                 /* result rows streamed */
    uint64_t hash;                 /* hash of every streamed row's columns */
    uint64_t est_bytes;
    double t_arrival, t_admit, t_summary, t_chunk, t_last;   /* t_chunk: first chunk out */
} gj_request_result;
typedef struct {
    int32_t peak_in_flight;
    uint64_t peak_admitted_bytes;
    double wall_s;
} gj_server_stats;
gj_status gj_server_create(gj_ctx *ctx, int32_t n_slots, uint64_t hbm_budget, uint64_t chunk_rows,
                           uint64_t max_rows, gj_server **out);
gj_status gj_server_run(gj_server *server, int32_t n_requests, const int32_t *rel_ids,
                        const int32_t *query_off, const double *arrival_offsets,
                        gj_request_result *results, gj_server_stats *stats);
void gj_server_destroy(gj_server *server);

/*
 * Row-sharded counting pass: one rank's part, for a query whose relations
 * are each split by rows across ranks (each rank loads its rows and creates
 * the query as usual).  No counterpart in the paper's single-machine
 * setting; it rests on Algorithm 2's sum-out being a sum (Section 3.3): a
 * message summed over all rows is the sum of the ranks' partial messages,
 * given the children's global messages.  Every separator must be one
 * attribute.  Relations are indexed by query position; "children" are a
 * relation's children in the join tree in position order (the parents are
 * those of gj_query_sizes).  A message to relation rel's parent is a dense
 * uint64 vector over rel's separator value domain [lo, lo + len), the same
 * on every rank; entries saturate at UINT64_MAX like the summary.
 *
 * gj_shard_domain: the range [*lo, *hi] of rel's separator attribute over
 * this rank's rows of rel and of its parent (*lo > *hi when both are
 * empty); the ranks agree on the union.  rel must not be the root.
 * gj_shard_up: rel's partial message from this rank's rows, given the
 * children's global messages (child_msg[c] over [child_lo[c],
 * child_lo[c] + child_len[c]), device arrays): msg_out[v - lo] (device,
 * len entries) = sum over rel's local groups with separator value v of
 * cnt * prod_c child_msg[c][key_c - child_lo[c]].  For the root, lo and
 * len are ignored and msg_out[0] is the rank's partial join size.
 * gj_shard_down: given rel's global down message (down_in over [down_lo,
 * down_lo + down_len); NULL for the root) and the children's global
 * messages, child_down_out[c] (device, child_len[c] entries) = this rank's
 * partial down message to child c, and mult_out[g] (device, one entry per
 * local group in factor order, gj_query_sizes' n_groups[rel]) = the
 * local groups' partial multiplicities w * down.
 * All three return GJ_ERR_INVALID for a cyclic query, a separator of
 * several attributes or missing arrays; up and down wait for their stream.
 */
gj_status gj_shard_domain(gj_query *q, int32_t rel, int32_t *lo, int32_t *hi);
gj_status gj_shard_up(gj_query *q, int32_t rel, const uint64_t *const *child_msg,
                      const int32_t *child_lo, const int64_t *child_len, uint64_t *msg_out,
                      int32_t lo, int64_t len);
gj_status gj_shard_down(gj_query *q, int32_t rel, const uint64_t *down_in, int32_t down_lo,
                        int64_t down_len, const uint64_t *const *child_msg,
                        const int32_t *child_lo, const int64_t *child_len,
                        uint64_t *const *child_down_out, uint64_t *mult_out);

/*
 * Factor construction without any device allocation.  The paper has no
 * counterpart; this exists for callers that cannot allocate device memory:
 * a database engine or serving process that hands all device memory to its
 * own pool (where cudaMalloc would fail or break the pool's accounting), or
 * code on a latency-critical path where cudaMalloc/cudaFree would
 * synchronise the device.
 *
 * Same result as gj_build_factors + gj_factor_export for `col_order`
 * (NULL = declared order): perm_dev (uint32[n_rows]), gstart_dev (capacity
 * n_rows + 1 entries; n_groups + 1 are written), gkey_dev (capacity
 * n_keys * n_rows; column c of group g at gkey[c*n_groups + g]) and
 * *n_groups.  key_cols is a host array of n_keys device pointers.  Work is
 * enqueued on `cuda_stream` on `device`.  Every call waits for that stream
 * before it returns: it reads the key ranges, the group count and the
 * device error word back into host memory.  So no call can be captured
 * into a CUDA graph: on a capturing stream the synchronisation fails and
 * invalidates the capture.
 *
 * All scratch lives in one fixed device array inside the library (about
 * 6.7 MB, held on every device that loads the library until the process
 * exits), so n_rows may not exceed GJ_NOALLOC_MAX_ROWS: larger inputs return
 * GJ_ERR_INVALID before any work is enqueued.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress).  Every call
 * shares the array and keeps its last contents: calls whose work overlaps on
 * the GPU (other streams, other threads) race and must be serialised by the
 * caller.
 */
#define GJ_NOALLOC_MAX_ROWS (1 << 18)
gj_status gj_factor_build_noalloc(int32_t device, void *cuda_stream, int64_t n_rows,
                                  int32_t n_keys, const int32_t *const *key_cols,
                                  const int32_t *col_order, uint32_t *perm_dev,
                                  uint32_t *gstart_dev, int32_t *gkey_dev, int64_t *n_groups);

#ifdef __cplusplus
}
#endif

#endif /* GJ_H */
