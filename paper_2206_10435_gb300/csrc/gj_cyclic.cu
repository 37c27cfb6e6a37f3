// gj_cyclic.cu -- cyclic queries in general (Sections 3.2.1 and 3.4).
//
// A query whose relation order gives no join tree is answered over a
// junction tree: two maxcliques where the second can be built as below
// (cyc_split), else one maxclique holding every attribute.  A clique's
// potential (Algorithm 1: the relations' potentials joined, frequencies
// multiplied) is built at the level of groups (distinct key tuples),
// relation by relation in query order:
//
//   items_0 = every group of relation 0
//   items_j = { (g_0..g_j-1, g) : g a group of relation j whose values of
//               the attributes j shares with relations 0..j-1 equal the
//               item's }
//
// Relation j's factor is ordered by those shared columns first, so the
// matching groups of an item are one contiguous range, found by two binary
// searches (or read off a table over the shared values); inside it the
// groups follow j's new attributes in V order.  So
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

// the two-clique plan (cyc_split below): every item of the second clique
// packed into one word over its attributes' values (fields from the low
// end: field f at shift[f]); vals = the item's index
struct ItemPack {
    int nf;
    const int32_t *key[8];      // group keys of the attribute's holder
    const uint32_t *grp[8];     // the items' groups of that holder
    int32_t mn[8];
    int shift[8];
};

__global__ void k_cyc_pack_items(ItemPack p, int64_t n, uint64_t *keys, uint32_t *vals) {
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < n; i += (int64_t)gridDim.x * CT) {
        uint64_t w = 0;
        for (int f = 0; f < p.nf; f++)
            w |= (uint64_t)((uint32_t)p.key[f][p.grp[f][i]] - (uint32_t)p.mn[f]) << p.shift[f];
        keys[i] = w;
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_cyc_gather(int64_t n, const uint32_t *__restrict__ src, const uint32_t *__restrict__ idx,
                             uint32_t *dst) {
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < n; i += (int64_t)gridDim.x * CT)
        dst[i] = src[idx[i]];
}

__global__ void k_cyc_item_vals(int64_t n, const int32_t *__restrict__ key, const uint32_t *__restrict__ grp,
                                int32_t *dst) {
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < n; i += (int64_t)gridDim.x * CT)
        dst[i] = key[grp[i]];
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

// A step's optional table over the values of its first one or two shared
// columns: their minima and value counts (n = 0: no table).
struct RangeInfo {
    int n = 0;
    int32_t mn[2] = {0, 0};
    int64_t nv[2] = {0, 0};
};

inline cudaError_t first_error(cudaError_t e) { return e != cudaSuccess ? e : cudaGetLastError(); }

// One step of the group-wise join: the F items (their groups by item
// position in cur[0 .. s.j - 1]) joined with the s.G candidates of position
// s.j.  On success cur holds the new items (s.j + 1 arrays) and F their
// number; GJ_ERR_OOM when they would be more than 2^31 or memory runs out.
// Every array of the step is freed on every way out.
gj_status cyc_step(Ctx &c, StepSpec s, const RangeInfo &ri, std::vector<uint32_t *> &cur, int64_t &F) {
    constexpr int64_t MAX_RANGE = 1ll << 24;
    Temps tmp(c);
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t x) {
        note_cuda_error(x, __FILE__, __LINE__);
        return x == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
    };
    s.err = c.err;
    for (int p = 0; p < s.j; p++) s.item_grp[p] = cur[p];
    uint64_t *cnt = nullptr, *excl = nullptr, *tot = nullptr;
    uint32_t *lo = nullptr;
    if ((e = tmp.alloc(&cnt, F)) != cudaSuccess || (e = tmp.alloc(&excl, F)) != cudaSuccess ||
        (e = tmp.alloc(&lo, F)) != cudaSuccess || (e = tmp.alloc(&tot, 1)) != cudaSuccess)
        return fail(e);
    int rc = std::min(ri.n, 2);
    if (rc == 2 && ri.nv[0] * ri.nv[1] > MAX_RANGE) rc = 1;
    if (rc == 1 && ri.nv[0] > MAX_RANGE) rc = 0;
    if (s.G > 0 && rc > 0) {
        const int64_t nx = rc == 2 ? ri.nv[0] * ri.nv[1] : ri.nv[0];
        s.range_cols = rc;
        for (int ci = 0; ci < rc; ci++) {
            s.range_mn[ci] = ri.mn[ci];
            s.range_nv[ci] = (uint32_t)ri.nv[ci];
        }
        uint32_t *rl = nullptr;
        if ((e = tmp.alloc(&rl, nx + 1)) != cudaSuccess) return fail(e);
        k_cyc_ranges<<<grid_of(c, nx + 1), CT, 0, c.stream>>>(s, nx, rl); c.launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
        s.range_lo = rl;
    }
    uint64_t Fout = 0;
    if (F > 0) {
        k_cyc_count<<<grid_of(c, F), CT, 0, c.stream>>>(s, F, cnt, lo); c.launches++;
        if ((e = first_error(cudaSuccess)) != cudaSuccess ||
            (e = scan_u64_sat(c, cnt, nullptr, excl, F, tot, nullptr, nullptr)) != cudaSuccess ||
            (e = read_u64(c, tot, &Fout)) != cudaSuccess)
            return fail(e);
    }
    if (Fout > 0x7fffffffull) return GJ_ERR_OOM;   // more partial blocks than this path holds
    std::vector<uint32_t *> nxt(s.j + 1, nullptr);
    for (int p = 0; p <= s.j; p++)
        if ((e = tmp.alloc(&nxt[p], (int64_t)Fout)) != cudaSuccess) return fail(e);
    if (Fout > 0) {
        OutGrp og{};
        for (int p = 0; p <= s.j; p++) og.g[p] = nxt[p];
        uint32_t *tf = nullptr;
        const int64_t tiles = ((int64_t)Fout + WT - 1) / WT;
        if ((e = tmp.alloc(&tf, tiles)) != cudaSuccess) return fail(e);
        k_cyc_tile_first<<<grid_of(c, F), CT, 0, c.stream>>>(F, cnt, excl, tf); c.launches++;
        k_cyc_write<<<grid_of(c, (int64_t)Fout), CT, 0, c.stream>>>(s, F, excl, lo, (int64_t)Fout, tf, og); c.launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    }
    for (uint32_t *g : nxt) tmp.keep(g);
    for (auto &g : cur) dfree(c, g);
    cur = nxt;
    F = (int64_t)Fout;
    return GJ_OK;
}

// The step adding relation j of the query to items over relations 0..j-1
// (every shared attribute).
StepSpec relation_step(QueryState &q, int j, RangeInfo &ri) {
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
    ri = RangeInfo{};
    ri.n = std::min(2, s.nshared);
    for (int ci = 0; ci < ri.n; ci++) {
        const int col = t.sep_cols[ci];
        ri.mn[ci] = t.R->kmin[col];
        ri.nv[ci] = (int64_t)t.R->kmax[col] - (int64_t)t.R->kmin[col] + 1;
    }
    return s;
}

// The junction tree with two maxcliques, for queries of four or more
// relations: clique 1 holds the attributes of relations 0 and 1, clique 2
// those of relations 2 .. k-1, the separator their common attributes S (for
// the 4-cycle R0(A,B) R1(B,C) R2(C,D) R3(D,A): cliques {A,B,C} and {C,D,A},
// S = {A,C}, the chord A-C of its triangulation, Section 2.2).  Each
// clique's potential is built group-wise as on one clique; clique 2's items
// are then sorted by S (in V order) and the rest of its attributes (in V
// order), and joined with clique 1's items on S.  No item ever spans both
// sides before the join, so the paths a single clique would materialise
// (every 3-path of a 4-cycle) never appear.  The blocks come out in V order:
// clique 1's items in V order, each one's matches in the order of clique
// 2's other attributes.  Taken when every relation of clique 2 after the
// first shares an attribute with the earlier ones of its clique (plan_cyclic
// orders its factor by those columns first), S is not empty, and clique 2's
// attributes pack into one 64-bit word; otherwise the query stays on one
// clique (applied = false).
gj_status cyc_split(QueryState &q, std::vector<uint32_t *> &blocks, int64_t &nb, bool &applied) {
    applied = false;
    const int k = q.k;
    if (k < 4) return GJ_OK;
    Ctx &c = q.ctx();
    auto col_of = [&](int j, int32_t a) {
        for (int cc = 0; cc < q.r[j].R->nk; cc++)
            if (q.r[j].R->attr[cc] == a) return cc;
        return -1;
    };
    auto holder = [&](int32_t a, int j0, int j1) {   // first relation of [j0, j1) holding a
        for (int j = j0; j < j1; j++)
            if (col_of(j, a) >= 0) return j;
        return -1;
    };
    // S and clique 2's other attributes, both in V order
    std::vector<int32_t> S, N;
    for (size_t v = 0; v < q.var_rel.size(); v++) {
        const int32_t a = q.r[q.var_rel[v]].R->attr[q.var_col[v]];
        if (holder(a, 2, k) < 0) continue;
        (holder(a, 0, 2) >= 0 ? S : N).push_back(a);
    }
    if (S.empty() || S.size() + N.size() > 8) return GJ_OK;
    // clique 2's cascade: relation j joins relations 2..j-1 on a leading run
    // of its shared columns
    std::vector<int> lead(k, 0);
    for (int j = 3; j < k; j++) {
        const QRel &t = q.r[j];
        int m = 0;
        while (m < (int)t.sep_cols.size() && holder(t.R->attr[t.sep_cols[m]], 2, j) >= 0) m++;
        for (int ci = m; ci < (int)t.sep_cols.size(); ci++)
            if (holder(t.R->attr[t.sep_cols[ci]], 2, j) >= 0) return GJ_OK;
        if (m == 0) return GJ_OK;
        lead[j] = m;
    }
    // the sort key of clique 2's items: S then N, least significant last
    ItemPack ip{};
    std::vector<int32_t> fields(S);
    fields.insert(fields.end(), N.begin(), N.end());
    std::vector<int> fh(fields.size()), fc(fields.size());
    int bits = 0;
    for (int f = (int)fields.size() - 1; f >= 0; f--) {
        fh[f] = holder(fields[f], 2, k);
        fc[f] = col_of(fh[f], fields[f]);
        const Relation &R = *q.r[fh[f]].R;
        const uint32_t range = (uint32_t)((int64_t)R.kmax[fc[f]] - (int64_t)R.kmin[fc[f]]);
        const int b = range == 0 ? 0 : 32 - __builtin_clz(range);
        ip.shift[f] = bits;
        ip.mn[f] = R.kmin[fc[f]];
        bits += b;
    }
    if (bits > 64) return GJ_OK;
    applied = true;

    std::vector<uint32_t *> A(1, nullptr), Bi(1, nullptr), Bs;
    std::vector<int32_t *> vS;
    uint64_t *keys = nullptr;
    uint32_t *vals = nullptr;
    auto free_all = [&]() {
        for (auto &g : A) dfree(c, g);
        for (auto &g : Bi) dfree(c, g);
        for (auto &g : Bs) dfree(c, g);
        for (auto &v : vS) dfree(c, v);
        dfree(c, keys);
        dfree(c, vals);
    };
    auto cuda_fail = [&](cudaError_t x) {
        note_cuda_error(x, __FILE__, __LINE__);
        free_all();
        return x == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
    };
    cudaError_t e = cudaSuccess;
    gj_status st = GJ_OK;
    // clique 1: relations 0 and 1
    int64_t FA = q.r[0].F->G, FB = q.r[2].F->G;
    if ((e = dalloc(c, &A[0], FA)) != cudaSuccess) return cuda_fail(e);
    if (FA > 0) { k_cyc_iota<<<grid_of(c, FA), CT, 0, c.stream>>>(A[0], FA); c.launches++; }
    {
        RangeInfo ri;
        StepSpec s1 = relation_step(q, 1, ri);
        if ((st = cyc_step(c, s1, ri, A, FA)) != GJ_OK) { free_all(); return st; }
    }
    // clique 2: relations 2 .. k-1, at item positions 0 .. k-3
    if ((e = dalloc(c, &Bi[0], FB)) != cudaSuccess) return cuda_fail(e);
    if (FB > 0) { k_cyc_iota<<<grid_of(c, FB), CT, 0, c.stream>>>(Bi[0], FB); c.launches++; }
    for (int j = 3; j < k; j++) {
        const QRel &t = q.r[j];
        StepSpec sb{};
        sb.j = j - 2;
        sb.nshared = lead[j];
        RangeInfo ri;
        ri.n = std::min(2, sb.nshared);
        for (int ci = 0; ci < sb.nshared; ci++) {
            const int32_t a = t.R->attr[t.sep_cols[ci]];
            const int h = holder(a, 2, j);
            sb.src_key[ci] = q.r[h].F->gkey + (int64_t)col_of(h, a) * q.r[h].F->G;
            sb.src_pos[ci] = h - 2;
            sb.dst_key[ci] = t.F->gkey + (int64_t)t.sep_cols[ci] * t.F->G;
            if (ci < 2) {
                ri.mn[ci] = t.R->kmin[t.sep_cols[ci]];
                ri.nv[ci] = (int64_t)t.R->kmax[t.sep_cols[ci]] - (int64_t)t.R->kmin[t.sep_cols[ci]] + 1;
            }
        }
        sb.G = t.F->G;
        if ((st = cyc_step(c, sb, ri, Bi, FB)) != GJ_OK) { free_all(); return st; }
    }
    // clique 2's items in (S, N) order
    Bs.assign(k - 2, nullptr);
    if ((e = dalloc(c, &keys, FB)) != cudaSuccess || (e = dalloc(c, &vals, FB)) != cudaSuccess)
        return cuda_fail(e);
    for (int p = 0; p < k - 2; p++)
        if ((e = dalloc(c, &Bs[p], FB)) != cudaSuccess) return cuda_fail(e);
    if (FB > 0) {
        ip.nf = (int)fields.size();
        for (int f = 0; f < ip.nf; f++) {
            ip.key[f] = q.r[fh[f]].F->gkey + (int64_t)fc[f] * q.r[fh[f]].F->G;
            ip.grp[f] = Bi[fh[f] - 2];
        }
        k_cyc_pack_items<<<grid_of(c, FB), CT, 0, c.stream>>>(ip, FB, keys, vals); c.launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
        if (bits > 0 && (e = radix_sort_u64_u32(c, keys, vals, FB, bits)) != cudaSuccess) return cuda_fail(e);
        for (int p = 0; p < k - 2; p++) {
            k_cyc_gather<<<grid_of(c, FB), CT, 0, c.stream>>>(FB, Bi[p], vals, Bs[p]); c.launches++;
        }
    }
    dfree(c, keys);
    for (auto &g : Bi) dfree(c, g);
    Bi.clear();
    // S's values of the sorted items, the join's keys on clique 2's side
    vS.assign(S.size(), nullptr);
    for (size_t f = 0; f < S.size(); f++) {
        if ((e = dalloc(c, &vS[f], FB)) != cudaSuccess) return cuda_fail(e);
        if (FB > 0) {
            k_cyc_item_vals<<<grid_of(c, FB), CT, 0, c.stream>>>(
                FB, q.r[fh[f]].F->gkey + (int64_t)fc[f] * q.r[fh[f]].F->G, Bs[fh[f] - 2], vS[f]); c.launches++;
        }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    // the join of the cliques on S: clique 1's items (positions 0, 1) with
    // the sorted items of clique 2 (position 2: the item's index)
    {
        StepSpec sf{};
        sf.j = 2;
        sf.nshared = (int)S.size();
        RangeInfo ri;
        ri.n = std::min<int>(2, sf.nshared);
        for (int f = 0; f < sf.nshared; f++) {
            const int h = holder(S[f], 0, 2);
            sf.src_key[f] = q.r[h].F->gkey + (int64_t)col_of(h, S[f]) * q.r[h].F->G;
            sf.src_pos[f] = h;
            sf.dst_key[f] = vS[f];
            if (f < 2) {
                ri.mn[f] = ip.mn[f];
                ri.nv[f] = (int64_t)q.r[fh[f]].R->kmax[fc[f]] - (int64_t)ip.mn[f] + 1;
            }
        }
        sf.G = FB;
        if ((st = cyc_step(c, sf, ri, A, FA)) != GJ_OK) { free_all(); return st; }
    }
    // the blocks' groups by relation
    blocks.assign(k, nullptr);
    blocks[0] = A[0];
    blocks[1] = A[1];
    A[0] = A[1] = nullptr;
    for (int p = 0; p < k - 2; p++) {
        if ((e = dalloc(c, &blocks[2 + p], FA)) != cudaSuccess) {
            for (auto &g : blocks) dfree(c, g);
            return cuda_fail(e);
        }
        if (FA > 0) { k_cyc_gather<<<grid_of(c, FA), CT, 0, c.stream>>>(FA, Bs[p], A[2], blocks[2 + p]); c.launches++; }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) {
        for (auto &g : blocks) dfree(c, g);
        return cuda_fail(e);
    }
    free_all();
    nb = FA;
    return GJ_OK;
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
// Factor orders: shared columns first (declared order; from relation 3 on,
// those shared with relations 2..j-1 ahead of the others), then the rest;
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
        if (j >= 3 && k >= 4) {
            // shared columns whose attribute relations 2..j-1 hold come
            // first (stable): the factor is then ordered so that the second
            // clique of cyc_split can join relation j on a leading run
            auto in_second = [&](int c) {
                for (int i = 2; i < j; i++)
                    for (int cc = 0; cc < q.r[i].R->nk; cc++)
                        if (q.r[i].R->attr[cc] == t.R->attr[c]) return true;
                return false;
            };
            std::vector<int> order(t.sep_cols.size());
            for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
            std::stable_partition(order.begin(), order.end(), [&](int i) { return in_second(t.sep_cols[i]); });
            std::vector<int> sc, sr, sl;
            for (int i : order) {
                sc.push_back(t.sep_cols[i]);
                sr.push_back(t.cyc_src_rel[i]);
                sl.push_back(t.cyc_src_col[i]);
            }
            t.sep_cols = sc;
            t.cyc_src_rel = sr;
            t.cyc_src_col = sl;
        }
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
        int64_t F = 0;
        bool split = false;
        gj_status sst = cyc_split(q, cur, F, split);
        if (sst != GJ_OK) return sst;
        if (!split) {
            // one clique: items of relation 0 (all its groups), then every
            // relation in query order
            F = q.r[0].F->G;
            TRY(dalloc(c, &cur[0], F));
            if (F > 0) { k_cyc_iota<<<grid_of(c, F), CT, 0, c.stream>>>(cur[0], F); c.launches++; }
            TRY(cudaGetLastError());
            for (int j = 1; j < k; j++) {
                RangeInfo ri;
                StepSpec s = relation_step(q, j, ri);
                gj_status st = cyc_step(c, s, ri, cur, F);
                if (st != GJ_OK) {
                    for (auto &g : cur) dfree(c, g);
                    return st;
                }
            }
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
