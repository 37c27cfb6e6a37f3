// gj_cyclic.cu -- cyclic queries in general (Sections 3.2.1 and 3.4).
//
// A query whose relation order gives no join tree is answered over a
// junction tree.  Here it is the junction tree of one maxclique holding
// every attribute: its potential (Algorithm 1: the relations' potentials
// joined, frequencies multiplied) is built at the level of groups (distinct
// key tuples), relation by relation in query order:
//
//   items_0 = every group of relation 0
//   items_j = { (g_0..g_j-1, g) : g a group of relation j whose values of
//               the attributes j shares with relations 0..j-1 equal the
//               item's }
//
// Relation j's factor is ordered by those shared columns first, so the
// matching groups of an item are one contiguous range, found by two binary
// searches; inside it the groups follow j's new attributes in V order.  So
// the final items (the blocks: one group per relation, consistent on every
// shared attribute) come out in V order with no sort, V being the
// attributes in order of first appearance.  A block stands for the
// Cartesian product of its groups' rows, prod_j cnt_j rows in the mixed
// radix of the row ids (relation k-1 fastest); the exclusive scan of the
// block sizes places every block in the result, and the emit kernel of the
// acyclic path expands any window of rows from the blocks.  The 3-cycle has
// its own path (gj_cycle.cu), which never forms the intermediate pairs.
#include <string.h>

#include <algorithm>

#include "gj_emit.cuh"

namespace gj {

gj_status check_device_error(Ctx &c);
bool make_emit_spec(QueryState &q, void *const *out_cols, uint32_t *const *rowid_cols,
                    const uint32_t *const *grp, const uint64_t *A, Emit4Spec &s);
void note_cuda_error(cudaError_t e, const char *file, int line);

namespace {

constexpr int CT = 256;

// Where step j finds the values of its shared attributes: for the c-th
// shared column of relation j (in its factor order), the group keys of the
// relation that first holds the attribute, at that relation's group in the
// item.
struct StepSpec {
    int j;                          // relation added by this step
    int nshared;
    const int32_t *src_key[MAX_KEYS];   // holder's group keys of the attribute
    int src_pos[MAX_KEYS];              // holder's position in the item
    const int32_t *dst_key[MAX_KEYS];   // relation j's group keys of the attribute
    int64_t G;                          // relation j's groups
    const uint32_t *item_grp[MAX_REL];  // the items' groups, by relation
    // optional: a table over the first range_cols (1 or 2) shared columns'
    // values: the groups whose values are range_mn[c] + v_c are
    // [range_lo[x], range_lo[x + 1]), x = v_0 (* range_nv[1] + v_1); when
    // the table covers every shared column that range is the answer, else
    // the searches run inside it
    const uint32_t *range_lo;
    int range_cols;
    int32_t range_mn[2];
    uint32_t range_nv[2];
    uint32_t *err;
};

// compares relation j's group g with the item's values (lexicographic over
// the shared columns in factor order)
__device__ __forceinline__ int cmp_group(const StepSpec &s, const int32_t (&want)[MAX_KEYS], int64_t g) {
    for (int c = 0; c < s.nshared; c++) {
        const int32_t v = s.dst_key[c][g];
        if (v != want[c]) return v < want[c] ? -1 : 1;
    }
    return 0;
}

// range_lo of a step: relation j's groups are sorted by their shared columns
// first, so range_lo[x] is the first group whose leading range_cols values
// are >= the tuple that x encodes (one binary search per x; x = the table's
// size gives G)
__global__ void k_cyc_ranges(StepSpec s, int64_t nx, uint32_t *lo) {
    for (int64_t x = (int64_t)blockIdx.x * CT + threadIdx.x; x <= nx; x += (int64_t)gridDim.x * CT) {
        int32_t want[2] = {0, 0};
        if (s.range_cols == 2) {
            want[0] = s.range_mn[0] + (int32_t)(x / s.range_nv[1]);
            want[1] = s.range_mn[1] + (int32_t)(x % s.range_nv[1]);
        } else {
            want[0] = s.range_mn[0] + (int32_t)x;
        }
        int64_t a = 0, b = s.G;
        if (x < nx) {
            while (a < b) {
                const int64_t m = (a + b) >> 1;
                int cmp = 0;
                for (int c = 0; c < s.range_cols && cmp == 0; c++) {
                    const int32_t v = s.dst_key[c][m];
                    cmp = v < want[c] ? -1 : (v > want[c] ? 1 : 0);
                }
                if (cmp < 0) a = m + 1; else b = m;
            }
        } else {
            a = s.G;
        }
        lo[x] = (uint32_t)a;
    }
}

__global__ void k_cyc_count(StepSpec s, int64_t F, uint64_t *cnt, uint32_t *lo_out) {
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < F; i += (int64_t)gridDim.x * CT) {
        int32_t want[MAX_KEYS];
        for (int c = 0; c < s.nshared; c++) want[c] = s.src_key[c][s.item_grp[s.src_pos[c]][i]];
        int64_t a = 0, hi = s.G;
        if (s.range_lo) {
            int64_t x = 0;
            bool none = false;   // a value outside the relation's range: no group
            for (int c = 0; c < s.range_cols; c++) {
                const int64_t v = (int64_t)want[c] - (int64_t)s.range_mn[c];
                none |= v < 0 || v >= (int64_t)s.range_nv[c];
                x = x * (int64_t)s.range_nv[c] + v;
            }
            if (none) {
                cnt[i] = 0;
                lo_out[i] = 0;
                continue;
            }
            a = s.range_lo[x];
            hi = s.range_lo[x + 1];
            if (s.range_cols == s.nshared) {   // the table's range is the answer
                cnt[i] = (uint64_t)(hi - a);
                lo_out[i] = (uint32_t)a;
                continue;
            }
        }
        int64_t b = hi;           // first group >= want
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (cmp_group(s, want, m) < 0) a = m + 1; else b = m;
        }
        const int64_t lo = a;
        b = hi;                   // first group > want
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (cmp_group(s, want, m) <= 0) a = m + 1; else b = m;
        }
        cnt[i] = (uint64_t)(a - lo);
        lo_out[i] = (uint32_t)lo;
    }
}

struct OutGrp {
    uint32_t *g[MAX_REL];
};

// tile_first[t] = the item owning output slot t * WT (an item owns slots
// [excl, excl + cnt)); one scatter over the items with slots
constexpr int64_t WT = 1024;

__global__ void k_cyc_tile_first(int64_t F, const uint64_t *__restrict__ cnt,
                                 const uint64_t *__restrict__ excl, uint32_t *tile_first) {
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < F; i += (int64_t)gridDim.x * CT) {
        const uint64_t c = cnt[i];
        if (c == 0) continue;
        const uint64_t lo = excl[i], hi = lo + c;
        for (uint64_t t = (lo + WT - 1) / WT; t * WT < hi; t++) tile_first[t] = (uint32_t)i;
    }
}

// output slot o belongs to the last item whose exclusive offset is <= o;
// searched between the owners of its tile's first slot and of the next
// tile's (items without slots lie between them too)
__global__ void k_cyc_write(StepSpec s, int64_t F, const uint64_t *__restrict__ excl,
                            const uint32_t *__restrict__ lo_in, int64_t Fout,
                            const uint32_t *__restrict__ tile_first, OutGrp out) {
    const int64_t tiles = (Fout + WT - 1) / WT;
    for (int64_t o = (int64_t)blockIdx.x * CT + threadIdx.x; o < Fout; o += (int64_t)gridDim.x * CT) {
        const int64_t t = o / WT;
        int64_t a = tile_first[t], b = t + 1 < tiles ? (int64_t)tile_first[t + 1] + 1 : F;
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (excl[m] <= (uint64_t)o) a = m + 1; else b = m;
        }
        const int64_t i = a - 1;
        if (i < 0) { raise_err(s.err, ERRF_BOUNDS); continue; }
        for (int p = 0; p < s.j; p++) out.g[p][o] = s.item_grp[p][i];
        out.g[s.j][o] = lo_in[i] + (uint32_t)(o - (int64_t)excl[i]);
    }
}

struct SizeSpec {
    int k;
    const uint32_t *gstart[MAX_REL];
    const uint32_t *grp[MAX_REL];
};

// a block's rows: the product of its groups' counts (saturating)
__global__ void k_cyc_sizes(SizeSpec s, int64_t B, uint64_t *W) {
    for (int64_t b = (int64_t)blockIdx.x * CT + threadIdx.x; b < B; b += (int64_t)gridDim.x * CT) {
        uint64_t w = 1;
        for (int j = 0; j < s.k; j++) {
            const uint32_t g = s.grp[j][b];
            w = sat_mul(w, (uint64_t)(s.gstart[j][g + 1] - s.gstart[j][g]));
        }
        W[b] = w;
    }
}

__global__ void k_cyc_iota(uint32_t *g, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < n; i += (int64_t)gridDim.x * CT)
        g[i] = (uint32_t)i;
}

// the blocks overlapping result rows [row0, row_end): first and count
__global__ void k_cyc_window(const uint64_t *A, uint64_t B, uint64_t row0, uint64_t row_end,
                             uint32_t *out) {
    auto last_le = [&](uint64_t x) {
        uint64_t lo = 0, hi = B;
        while (lo < hi) {
            const uint64_t m = (lo + hi) >> 1;
            if (A[m] <= x) lo = m + 1; else hi = m;
        }
        return lo - 1;
    };
    const uint64_t f = last_le(row0), l = last_le(row_end - 1);
    out[0] = (uint32_t)f;
    out[1] = (uint32_t)(l - f + 1);
}

inline int grid_of(Ctx &c, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, CT), (int64_t)c.num_sms * 16));
}

cudaError_t read_u64(Ctx &c, const uint64_t *dev, uint64_t *host) {
    GJ_CUDA_TRY(cudaMemcpyAsync(c.pinned, dev, 8, cudaMemcpyDeviceToHost, c.stream));
    GJ_CUDA_TRY(cudaStreamSynchronize(c.stream));
    *host = c.pinned[0];
    return cudaSuccess;
}

}  // namespace

void cyc_free(Ctx &c, QueryState &q) {
    dfree(c, q.blk_A);
    for (auto &g : q.cyc_grp) dfree(c, g);
    q.cyc_grp.clear();
    q.nblocks = 0;
}

// The plan of a cyclic query (no join tree in this relation order): each
// relation after the first must share an attribute with those before it.
// Factor orders: shared columns first (declared order), then the others;
// V by first appearance.  False if the query is not of that form.
bool plan_cyclic(QueryState &q) {
    const int k = q.k;
    if (k < 2 || k > 8) return false;   // the emit kernel's templates
    std::vector<std::pair<int, int>> holder_of;   // by attribute: (relation, column)
    std::vector<int32_t> attrs;
    auto find = [&](int32_t a) {
        for (size_t i = 0; i < attrs.size(); i++)
            if (attrs[i] == a) return (int)i;
        return -1;
    };
    for (int j = 0; j < k; j++) {
        QRel &t = q.r[j];
        t.parent = -1;
        t.children.clear();
        t.sep_cols.clear();
        t.sep_cols_parent.clear();
        t.new_cols.clear();
        t.cyc_src_rel.clear();
        t.cyc_src_col.clear();
        for (int c = 0; c < t.R->nk; c++) {
            const int h = find(t.R->attr[c]);
            if (h >= 0 && j > 0) {
                t.sep_cols.push_back(c);
                t.cyc_src_rel.push_back(holder_of[h].first);
                t.cyc_src_col.push_back(holder_of[h].second);
            } else {
                t.new_cols.push_back(c);
            }
        }
        if (j > 0 && t.sep_cols.empty()) return false;   // a cross product
        if (j > 0) t.parent = t.cyc_src_rel[0];            // reported by gj_query_sizes
        for (int c = 0; c < t.R->nk; c++)
            if (find(t.R->attr[c]) < 0) {
                attrs.push_back(t.R->attr[c]);
                holder_of.emplace_back(j, c);
            }
    }
    q.cyc = true;
    q.pre.clear();
    q.pos.clear();
    for (int j = 0; j < k; j++) { q.pre.push_back(j); q.pos.push_back(j); }
    q.var_rel.clear();
    q.var_col.clear();
    for (int j = 0; j < k; j++)
        for (int c : q.r[j].new_cols) { q.var_rel.push_back(j); q.var_col.push_back(c); }
    q.col_rel.clear();
    q.col_pay.clear();
    for (int j = 0; j < k; j++)
        for (int p = 0; p < q.r[j].R->np; p++) { q.col_rel.push_back(j); q.col_pay.push_back(p); }
    return q.var_rel.size() <= 32 && q.col_rel.size() <= 32;
}

gj_status cyc_summarize(QueryState &q, uint64_t *total_out) {
    Ctx &c = q.ctx();
    cyc_free(c, q);
    q.summarized = false;
    const int k = q.k;
    cudaError_t e = cudaSuccess;
#define TRY(x)                                                 \
    do {                                                       \
        e = (x);                                               \
        if (e != cudaSuccess) {                                \
            note_cuda_error(e, __FILE__, __LINE__);            \
            goto fail;                                         \
        }                                                      \
    } while (0)
    std::vector<uint32_t *> cur(1, nullptr);   // the current items' groups, by relation
    {
        // items of relation 0: all its groups
        int64_t F = q.r[0].F->G;
        TRY(dalloc(c, &cur[0], F));
        if (F > 0) { k_cyc_iota<<<grid_of(c, F), CT, 0, c.stream>>>(cur[0], F); c.launches++; }
        TRY(cudaGetLastError());
        for (int j = 1; j < k && e == cudaSuccess; j++) {
            const QRel &t = q.r[j];
            StepSpec s{};
            s.j = j;
            s.nshared = (int)t.sep_cols.size();
            for (int ci = 0; ci < s.nshared; ci++) {
                const QRel &h = q.r[t.cyc_src_rel[ci]];
                s.src_key[ci] = h.F->gkey + (int64_t)t.cyc_src_col[ci] * h.F->G;
                s.src_pos[ci] = t.cyc_src_rel[ci];
                s.dst_key[ci] = t.F->gkey + (int64_t)t.sep_cols[ci] * t.F->G;
            }
            s.G = t.F->G;
            for (int p = 0; p < j; p++) s.item_grp[p] = cur[p];
            s.err = c.err;
            Temps tmp(c);
            uint64_t *cnt = nullptr, *excl = nullptr, *tot = nullptr;
            uint32_t *lo = nullptr;
            TRY(tmp.alloc(&cnt, F));
            TRY(tmp.alloc(&excl, F));
            TRY(tmp.alloc(&lo, F));
            TRY(tmp.alloc(&tot, 1));
            // a table over the value ranges of relation j's first one or
            // two shared columns, when it stays small (at most 2^24 entries)
            {
                constexpr int64_t MAX_RANGE = 1ll << 24;
                int64_t nv[2] = {0, 0};
                for (int ci = 0; ci < std::min(2, s.nshared); ci++) {
                    const int col = t.sep_cols[ci];
                    nv[ci] = (int64_t)t.R->kmax[col] - (int64_t)t.R->kmin[col] + 1;
                }
                int rc = std::min(2, s.nshared);
                if (rc == 2 && nv[0] * nv[1] > MAX_RANGE) rc = 1;
                if (rc == 1 && nv[0] > MAX_RANGE) rc = 0;
                if (t.F->G > 0 && rc > 0) {
                    const int64_t nx = rc == 2 ? nv[0] * nv[1] : nv[0];
                    s.range_cols = rc;
                    for (int ci = 0; ci < rc; ci++) {
                        s.range_mn[ci] = t.R->kmin[t.sep_cols[ci]];
                        s.range_nv[ci] = (uint32_t)nv[ci];
                    }
                    uint32_t *rl = nullptr;
                    TRY(tmp.alloc(&rl, nx + 1));
                    k_cyc_ranges<<<grid_of(c, nx + 1), CT, 0, c.stream>>>(s, nx, rl); c.launches++;
                    TRY(cudaGetLastError());
                    s.range_lo = rl;
                }
            }
            uint64_t Fout = 0;
            if (F > 0) {
                k_cyc_count<<<grid_of(c, F), CT, 0, c.stream>>>(s, F, cnt, lo); c.launches++;
                TRY(cudaGetLastError());
                TRY(scan_u64_sat(c, cnt, nullptr, excl, F, tot, nullptr, nullptr));
                TRY(read_u64(c, tot, &Fout));
            }
            if (Fout > 0x7fffffffull) {   // more partial blocks than this path holds
                for (auto &g : cur) dfree(c, g);
                return GJ_ERR_OOM;
            }
            std::vector<uint32_t *> nxt(j + 1, nullptr);
            bool ok = true;
            for (int p = 0; p <= j && ok; p++) ok = dalloc(c, &nxt[p], (int64_t)Fout) == cudaSuccess;
            if (!ok) {
                for (auto &g : nxt) dfree(c, g);
                for (auto &g : cur) dfree(c, g);
                return GJ_ERR_OOM;
            }
            if (Fout > 0) {
                OutGrp og{};
                for (int p = 0; p <= j; p++) og.g[p] = nxt[p];
                uint32_t *tf = nullptr;
                const int64_t tiles = ((int64_t)Fout + WT - 1) / WT;
                TRY(tmp.alloc(&tf, tiles));
                k_cyc_tile_first<<<grid_of(c, F), CT, 0, c.stream>>>(F, cnt, excl, tf); c.launches++;
                k_cyc_write<<<grid_of(c, (int64_t)Fout), CT, 0, c.stream>>>(s, F, excl, lo, (int64_t)Fout, tf, og); c.launches++;
            }
            for (auto &g : cur) dfree(c, g);
            cur = nxt;
            F = (int64_t)Fout;
            TRY(cudaGetLastError());
        }
        // blocks: their sizes, first rows and |Q|
        q.cyc_grp = cur;
        cur.clear();
        q.nblocks = (uint64_t)F;
        uint64_t total = 0;
        {
            Temps tmp(c);
            uint64_t *W = nullptr, *tot = nullptr;
            TRY(tmp.alloc(&W, F));
            TRY(tmp.alloc(&tot, 1));
            TRY(dalloc(c, &q.blk_A, F));
            if (F > 0) {
                SizeSpec ss{};
                ss.k = k;
                for (int j = 0; j < k; j++) { ss.gstart[j] = q.r[j].F->gstart; ss.grp[j] = q.cyc_grp[j]; }
                k_cyc_sizes<<<grid_of(c, F), CT, 0, c.stream>>>(ss, F, W); c.launches++;
                TRY(cudaGetLastError());
                TRY(scan_u64_sat(c, W, nullptr, q.blk_A, F, tot, nullptr, nullptr));
                TRY(read_u64(c, tot, &total));
            }
        }
        gj_status st = check_device_error(c);
        if (st != GJ_OK) return st;
        q.total = total;
        q.overflow = total == SAT;
        q.summarized = true;
        *total_out = total;
        return q.overflow ? GJ_ERR_OVERFLOW : GJ_OK;
    }
#undef TRY
fail:
    for (auto &g : cur) dfree(c, g);
    return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
}

gj_status cyc_desummarize(QueryState &q, uint64_t row0, uint64_t nrows, void *const *out_cols,
                          uint32_t *const *rowid_cols, uint64_t *n_out) {
    Ctx &c = q.ctx();
    *n_out = 0;
    if (!q.summarized) return GJ_ERR_STATE;
    if (q.overflow) return GJ_ERR_OVERFLOW;
    if (row0 >= q.total || nrows == 0) return GJ_OK;
    const uint64_t n = std::min<uint64_t>(nrows, q.total - row0);
    if (n > 0x7fffffffull || !out_cols) return GJ_ERR_INVALID;
    uint32_t *win = nullptr;
    if (dalloc(c, &win, 2) != cudaSuccess) return GJ_ERR_OOM;
    k_cyc_window<<<1, 1, 0, c.stream>>>(q.blk_A, q.nblocks, row0, row0 + n, win); c.launches++;
    uint32_t w[2] = {0, 0};
    gj_status st = GJ_OK;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(c.pinned, win, 8, cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
        cudaStreamSynchronize(c.stream) != cudaSuccess) {
        st = GJ_ERR_CUDA;
    } else {
        memcpy(w, c.pinned, 8);
        if ((uint64_t)w[0] + w[1] > q.nblocks || w[1] == 0) st = GJ_ERR_CUDA;   // the window lies inside |Q|
    }
    if (st == GJ_OK) {
        std::vector<const uint32_t *> grp(q.k);
        for (int j = 0; j < q.k; j++) grp[j] = q.cyc_grp[j] + w[0];
        Emit4Spec s{};
        if (!make_emit_spec(q, out_cols, rowid_cols, grp.data(), q.blk_A + w[0], s)) {
            st = GJ_ERR_INVALID;
        } else {
            cudaError_t e = launch_emit(c, q.k, s, win + 1, row0, (int64_t)n);
            if (c.prof) {   // the launcher recorded the start event
                uint64_t width = 4 * q.var_rel.size();
                for (size_t p = 0; p < q.col_rel.size(); p++) width += q.r[q.col_rel[p]].R->pw[q.col_pay[p]];
                cudaEventRecord(c.event(), c.stream);
                c.emit_launches++;
                c.emit_rows += n;
                c.emit_bytes += n * width;
            }
            st = e != cudaSuccess ? (e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA)
                                  : check_device_error(c);
        }
    }
    dfree(c, win);
    if (st == GJ_OK) *n_out = n;
    return st;
}

}  // namespace gj
