// gj_state.cuh -- host-side state of contexts, relations, factors, queries.
#pragma once

#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "gj_internal.cuh"

namespace gj {

constexpr int MAX_KEYS = 8;
constexpr int MAX_PAYLOADS = 8;
constexpr int MAX_REL = 16;

// Frequency table of one relation (Section 3.2), ordered by `order`
// (column indices, most significant first).  Rows of a group are contiguous
// in perm and in increasing row id.
struct Factor {
    std::vector<int> order;
    int64_t n = 0, G = 0;
    uint32_t *perm = nullptr;      // [n]
    uint32_t *gstart = nullptr;    // [G+1]
    int32_t *gkey = nullptr;       // [nk*G], declared column c at c*G
    std::vector<void *> pay;       // payloads in perm order (width*n bytes)
};

// Caller-supplied scratch of factor_build_in.
struct FactorScratch {
    uint64_t *keys, *k2;              // [n]
    uint32_t *v2;                     // [n]
    uint32_t *hist;                   // [8*256 + 8]
    unsigned long long *status;       // [status_tiles * 256]
    int64_t status_tiles;
    uint8_t *head;                    // [n]
    uint32_t *gid;                    // [n]
    uint32_t *gcount;                 // [1]
    void *scan_state;
    size_t scan_state_bytes;
    int32_t *mm;                      // [2 * MAX_KEYS]
};

struct Relation {
    int64_t n = 0;
    int nk = 0, np = 0;
    std::vector<int32_t> attr;
    std::vector<const int32_t *> key;
    std::vector<int32_t> pw;
    std::vector<const void *> pay;
    std::vector<void *> owned;     // library-owned copies
    bool have_minmax = false;
    std::vector<int32_t> kmin, kmax;
    std::map<std::vector<int>, std::unique_ptr<Factor>> factors;
};

struct CtxState {
    Ctx c;
    // guards the relation and factor maps (load, release, factor builds,
    // query planning); work on distinct queries does not take it
    std::recursive_mutex mu;
    std::map<int32_t, std::unique_ptr<Relation>> rels;
    int32_t next_id = 1;
};

// Per-relation state of a query: the relation's place in the join tree and
// its part of the summary.
struct QRel {
    int rel_id = 0;
    Relation *R = nullptr;
    Factor *F = nullptr;
    int parent = -1;                   // position in the query
    std::vector<int> children;         // positions, increasing
    std::vector<int> sep_cols;         // separator columns in this relation
    std::vector<int> sep_cols_parent;  // matching columns in the parent
    std::vector<int> new_cols;         // columns whose attribute the parent lacks
    // cyclic queries: for each shared column (sep_cols), the relation that
    // first holds its attribute and that relation's column
    std::vector<int> cyc_src_rel, cyc_src_col;
    // segments over the separator (non-root); their number S lives in
    // device memory (*S_dev), arrays are sized for G >= S
    uint32_t *S_dev = nullptr;
    uint32_t *seg_id = nullptr;        // [G]
    uint32_t *seg_first = nullptr;     // [S+1]
    // link to each child's segments: link[i][g] for children[i]
    std::vector<uint32_t *> link;
    // summary
    uint64_t *w = nullptr;             // [G]
    uint64_t *off = nullptr;           // [G] root: global offset; else rel_off
    uint64_t *msg = nullptr;           // [S] (non-root)
    uint64_t *down = nullptr;          // [S] (non-root)
    uint64_t *mult = nullptr;          // [G]
    // live (w > 0) groups, in group order; their number L is *L_dev
    uint32_t *L_dev = nullptr;
    uint32_t *lgid = nullptr;          // [L]
    uint64_t *loff = nullptr;          // [L]
    uint64_t *lw = nullptr;            // [L]
    uint32_t *lseg_first = nullptr;    // [S+1] (non-root)
};

struct QueryState {
    CtxState *cs = nullptr;
    // optional execution context of this query alone (own stream, readback
    // buffer and error word; shares the context's pool and factors)
    std::unique_ptr<Ctx> own;
    Ctx *exec = nullptr;               // own.get(), or a context lent by the server
    Ctx &ctx() { return exec ? *exec : cs->c; }
    int k = 0;
    std::vector<QRel> r;
    std::vector<int> pre;              // preorder of positions
    std::vector<int> pos;              // position -> preorder index
    std::vector<int> var_rel, var_col; // V
    std::vector<int> col_rel, col_pay; // payload output columns
    bool summarized = false;
    bool overflow = false;
    uint64_t total = 0;
    // one allocation holding every per-relation array of the summary (NULL
    // when they were allocated one by one: a loaded summary, or a serving
    // slot's arena)
    void *slab = nullptr;
    size_t slab_bytes = 0;
    // the cyclic 3-way join (gj_cycle.cu): key columns per relation
    // {shared with the previous relation, shared with the next} in the
    // cycle R0 -> R1 -> R2 -> R0, and its blocks (group triples) in result
    // order with their first rows
    bool tri = false;
    int tri_col[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    uint64_t nblocks = 0;
    uint64_t *blk_A = nullptr;
    uint32_t *blk_grp[3] = {nullptr, nullptr, nullptr};
    // a cyclic query answered over one maxclique (gj_cyclic.cu): its blocks'
    // groups, one array per relation (the first rows in blk_A, their number
    // in nblocks)
    bool cyc = false;
    std::vector<uint32_t *> cyc_grp;
    // relations (with their factors) owned by a summary loaded from a file
    std::vector<std::unique_ptr<Relation>> loaded;
};

}  // namespace gj

struct gj_ctx {
    gj::CtxState s;
};
struct gj_query {
    gj::QueryState s;
};
