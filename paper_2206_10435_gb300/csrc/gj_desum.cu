// gj_desum.cu -- desummarisation (Section 3.6) and summary levels (Def. 1).
//
// The summary places every key path (one group per relation, linked through
// the separators) at a known offset of the sorted result: the root group's
// off, plus, walking the relations in preorder, unit * rel_off of the chosen
// group, where unit is the number of result rows each "way" of that group
// stands for (the p_bucket * bucket product of Algorithm 4 times the ways of
// the subtrees still open beside it).  A window [row0, row0 + n) of the
// result is produced in two steps:
//
//   expand  Algorithm 4 restricted to the window, breadth first: a frontier
//           of path prefixes that overlap the window is extended one
//           relation at a time by the live groups of the linked segment that
//           overlap the window.  Each level is a count kernel, an exclusive
//           scan and a load-balanced write kernel (a CTA owns a tile of
//           output slots and maps them to prefixes by a shared-memory search),
//           so a segment with 10^5 groups costs no more than 10^5 tiny ones.
//   emit    every result row finds its block (full key path) by a binary
//           search of the block offsets staged in shared memory, splits its
//           offset inside the block into one row index per relation (mixed
//           radix, relation 1 most significant: rows of a block are ordered
//           by r_1..r_k) and writes the key values (block constants) and the
//           payloads, gathered from the factors' group-ordered copies.
//           Consecutive threads write consecutive rows of each column.
//
// A level of the paper's GFJS (Figure 2) is the run list of the frontier at
// the relation that introduces the level's variable.
#include <algorithm>

#include "gj_emit.cuh"

namespace gj {

gj_status check_device_error(Ctx &c);

namespace {

constexpr int DT = 256;          // threads per CTA
constexpr int EXP_TILE = 1024;   // output slots per CTA in expansion
constexpr int EMIT_TILE = 1024;  // result rows per CTA in emission

// One frontier: path prefixes (groups of preorder relations 0..depth-1).
// Arrays are sized for `cap` items; the item count lives in device memory.
struct Frontier {
    int64_t cap = 0;
    uint32_t *F_dev = nullptr;           // number of items
    uint64_t *A = nullptr;               // absolute first result row
    uint64_t *W = nullptr;               // product of the chosen groups' counts
    std::vector<uint32_t *> grp;         // grp[p][i]: group of preorder relation p
    uint32_t *lh = nullptr;              // live index of the last group (optional)
    uint64_t *unit = nullptr;            // rows per way of the last group (optional)
};

void frontier_free(Ctx &c, Frontier &f) {
    dfree(c, f.F_dev);
    dfree(c, f.A);
    dfree(c, f.W);
    for (auto &p : f.grp) dfree(c, p);
    f.grp.clear();
    dfree(c, f.lh);
    dfree(c, f.unit);
    f.cap = 0;
}

constexpr int MAXR = MAX_REL;

// Everything an expansion step needs, by value.
struct ExpandSpec {
    // relation being added (preorder index j)
    const uint32_t *link;          // parent's link to it, indexed by parent group
    int parent_p;                  // preorder index of its parent
    const uint32_t *lseg_first;    // [S+1]
    const uint64_t *msg;           // [S]
    const uint32_t *lgid;
    const uint64_t *loff;          // rel_off of live groups
    const uint64_t *lw;
    const uint32_t *gstart;
    // open subtrees beside it: multiply unit by their message
    int nrest;
    const uint32_t *rest_link[MAXR];
    const uint64_t *rest_msg[MAXR];
    int rest_parent_p[MAXR];
    // frontier in
    int depth;                     // = j
    const uint64_t *A, *W;
    const uint32_t *grp[MAXR];
    uint32_t *err;
};

__device__ __forceinline__ uint64_t item_unit(const ExpandSpec &s, int64_t i) {
    uint64_t u = s.W[i];
    for (int r = 0; r < s.nrest; r++) {
        uint32_t g = s.grp[s.rest_parent_p[r]][i];
        uint32_t seg = s.rest_link[r][g];
        u = sat_mul(u, seg == NONE ? 0ull : s.rest_msg[r][seg]);
    }
    return u;
}

// first h in [a, b) with key(h) > x, key non-decreasing
template <class F>
__device__ __forceinline__ uint32_t first_greater(uint32_t a, uint32_t b, uint64_t x, F key) {
    while (a < b) {
        uint32_t m = a + ((b - a) >> 1);
        if (key(m) > x) b = m; else a = m + 1;
    }
    return a;
}

__global__ void k_expand_count(ExpandSpec s, const uint32_t *F_dev, uint64_t row0, uint64_t row_end,
                               uint32_t *cnt, uint32_t *lo_out, uint64_t *unit_out,
                               uint32_t *err) {
    const int64_t F = *F_dev;
    for (int64_t i = (int64_t)blockIdx.x * DT + threadIdx.x; i < F; i += (int64_t)gridDim.x * DT) {
        uint32_t gp = s.grp[s.parent_p][i];
        uint32_t seg = s.link[gp];
        if (seg == NONE) { raise_err(err, ERRF_BOUNDS); cnt[i] = 0; lo_out[i] = 0; unit_out[i] = 1; continue; }
        uint64_t unit = item_unit(s, i);
        uint32_t a = s.lseg_first[seg], b = s.lseg_first[seg + 1];
        uint64_t A = s.A[i];
        uint32_t lo = a, hi = b;
        if (A < row0) {
            uint64_t X = (row0 - A) / unit;   // need unit * (off + w) > row0 - A
            lo = first_greater(a, b, X, [&](uint32_t h) { return s.loff[h] + s.lw[h]; });
        }
        uint64_t end = A + unit * s.msg[seg];
        if (end > row_end) {
            uint64_t Y = (row_end - 1 - A) / unit;   // need unit * off <= row_end - 1 - A
            hi = first_greater(a, b, Y, [&](uint32_t h) { return s.loff[h]; });
        }
        if (hi < lo) { raise_err(err, ERRF_BOUNDS); hi = lo; }
        cnt[i] = hi - lo;
        lo_out[i] = lo;
        unit_out[i] = unit;
    }
}

struct ExpandOut {
    uint64_t *A, *W;
    uint32_t *grp[MAXR];
    uint32_t *lh;
    uint64_t *unit;
    // last level of a desummarisation: tile_first[t] = block holding window
    // row t * tile_rows (the emit's tile map), written by the blocks
    uint32_t *tile_first;
    int64_t tile_rows, tiles;
    uint64_t row0;
    int64_t n;
};

// slot_first[t] = item owning output slot t*EXP_TILE (items own the slots
// [excl[i], excl[i] + cnt[i]) of the next frontier); one scatter pass.
__global__ void k_slot_first(const uint32_t *__restrict__ excl, const uint32_t *__restrict__ cnt,
                             const uint32_t *F_dev, uint32_t *slot_first) {
    const int64_t F = *F_dev;
    for (int64_t i = (int64_t)blockIdx.x * DT + threadIdx.x; i < F; i += (int64_t)gridDim.x * DT) {
        uint64_t lo = excl[i], hi = lo + cnt[i];
        for (uint64_t t = (lo + EXP_TILE - 1) / EXP_TILE; t * EXP_TILE < hi; t++)
            slot_first[t] = (uint32_t)i;
    }
}

// Tiles of EXP_TILE output slots, taken in turn by a persistent grid (the
// number of tiles follows from the next frontier's size in device memory);
// slot -> source item by a search of the item offsets staged in shared
// memory (each item has >= 1 slot).
__global__ void __launch_bounds__(DT)
k_expand_write(ExpandSpec s, const uint32_t *F_dev, const uint32_t *__restrict__ excl,
               const uint32_t *Fout_dev, const uint32_t *__restrict__ slot_first,
               const uint32_t *__restrict__ lo_in, const uint64_t *__restrict__ unit_in,
               ExpandOut o) {
    __shared__ uint32_t s_off[EXP_TILE + 1];
    __shared__ uint64_t s_A[EXP_TILE];   // tile map only: first rows of the tile's blocks
    __shared__ uint64_t s_end;            // and the end of its last block
    const int64_t F = *F_dev, Fout = *Fout_dev;
    const int64_t tiles = (Fout + EXP_TILE - 1) / EXP_TILE;
    const int j = s.depth;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t o0 = tile * EXP_TILE;
        const int64_t o1 = min(Fout, o0 + EXP_TILE);
        const int64_t first = slot_first[tile];
        const int64_t last = (tile + 1 < tiles) ? (int64_t)slot_first[tile + 1] : F - 1;
        const int nitems = (int)(last - first + 1);
        // every item owns >= 1 slot, so a tile sees at most EXP_TILE + 1 items
        if (last < first || nitems > EXP_TILE + 1) {
            if (threadIdx.x == 0) raise_err(s.err, ERRF_BOUNDS);
            return;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nitems; t += DT) s_off[t] = excl[first + t];
        __syncthreads();
        for (int64_t slot = o0 + threadIdx.x; slot < o1; slot += DT) {
            int a = 0, b = nitems;   // last t with s_off[t] <= slot
            while (a < b) { int m = (a + b) >> 1; if (s_off[m] <= (uint32_t)slot) a = m + 1; else b = m; }
            const int64_t i = first + a - 1;
            const uint32_t h = lo_in[i] + (uint32_t)(slot - s_off[a - 1]);
            const uint32_t g = s.lgid[h];
            const uint64_t unit = unit_in[i];
            const uint64_t A = s.A[i] + unit * s.loff[h];
            o.A[slot] = A;
            if (o.W) o.W[slot] = s.W[i] * (uint64_t)(s.gstart[g + 1] - s.gstart[g]);
            if (o.tile_first) {
                s_A[slot - o0] = A;
                // the tile's last block ends where the next tile starts: its
                // size is needed
                if (slot == o1 - 1) s_end = A + s.W[i] * (uint64_t)(s.gstart[g + 1] - s.gstart[g]);
            }
            for (int p = 0; p < j; p++) o.grp[p][slot] = s.grp[p][i];
            o.grp[j][slot] = g;
            if (o.lh) o.lh[slot] = h;
            if (o.unit) o.unit[slot] = unit;
        }
        if (o.tile_first) {
            // the tile's blocks hold rows [s_A[0], s_end) of the result: every
            // emit tile whose first row lies there points at the block holding
            // that row (threads take tiles, not blocks, so one huge block
            // costs no single thread more than its share)
            __syncthreads();
            const int64_t T = o.tile_rows;
            const int ns = (int)(o1 - o0);
            const uint64_t lo = s_A[0] > o.row0 ? s_A[0] - o.row0 : 0;
            const uint64_t hi = min(s_end - o.row0, (uint64_t)o.n);
            for (int64_t t = (int64_t)((lo + T - 1) / T) + threadIdx.x; t < o.tiles && (uint64_t)(t * T) < hi;
                 t += DT) {
                const uint64_t row = o.row0 + (uint64_t)(t * T);
                int a = 0, b = ns;   // last block with first row <= row
                while (a < b) { int m = (a + b) >> 1; if (s_A[m] <= row) a = m + 1; else b = m; }
                o.tile_first[t] = (uint32_t)(o0 + a - 1);
            }
        }
    }
}

// first index h in [a, b) with key(h) > x (key non-decreasing), by one warp:
// each round the 32 lanes probe 32 evenly spaced points and the interval
// shrinks to the gap between two of them (about log32 of the length rounds)
template <class F>
__device__ __forceinline__ uint32_t warp_first_greater(uint32_t a, uint32_t b, uint64_t x, F key) {
    const int lane = threadIdx.x & 31;
    while (b - a > 32) {
        const uint32_t step = (b - a + 31) / 32;
        const uint32_t p = a + lane * step;   // lane 0 probes a
        const bool gt = p < b && key(p) > x;
        const uint32_t m = __ballot_sync(0xffffffffu, gt);
        // the answer lies in (probe of the last lane not greater, probe of the first greater]
        const int f = m ? __ffs((int)m) - 1 : 32;   // first probing lane with key > x
        if (f == 0) return a;                        // key(a) > x
        if (f == 32) {                               // none greater: past the last probe inside
            a += ((b - 1 - a) / step) * step + 1;
        } else {                                     // between probes f - 1 and f
            b = a + (uint32_t)f * step;
            a += (uint32_t)(f - 1) * step + 1;
        }
    }
    const uint32_t p = a + lane;
    const bool gt = p < b && key(p) > x;
    const uint32_t m = __ballot_sync(0xffffffffu, gt);
    return m ? a + (uint32_t)(__ffs((int)m) - 1) : b;
}

__global__ void k_root_range(const uint64_t *loff, const uint64_t *lw, const uint32_t *L_dev,
                             uint64_t row0, uint64_t row_end, uint32_t *out, uint32_t *F_dev) {
    // live root groups h with [loff, loff + lw) overlapping [row0, row_end):
    // one warp, two searches
    const uint32_t L = *L_dev;
    const uint32_t lo = warp_first_greater(0u, L, row0, [&](uint32_t h) { return loff[h] + lw[h]; });
    const uint32_t hi = warp_first_greater(lo, L, row_end - 1, [&](uint32_t h) { return loff[h]; });
    if (threadIdx.x == 0) {
        out[0] = lo;
        out[1] = hi;
        *F_dev = hi - lo;
    }
}

__global__ void k_root_init(const uint32_t *lo_dev, const uint32_t *F_dev, const uint32_t *lgid,
                            const uint64_t *loff, const uint32_t *gstart, uint64_t *A, uint64_t *W,
                            uint32_t *grp0, uint32_t *lh, uint64_t *unit) {
    const uint32_t lo = *lo_dev;
    const int64_t F = *F_dev;
    for (int64_t i = (int64_t)blockIdx.x * DT + threadIdx.x; i < F; i += (int64_t)gridDim.x * DT) {
        uint32_t h = lo + (uint32_t)i;
        uint32_t g = lgid[h];
        A[i] = loff[h];
        W[i] = (uint64_t)(gstart[g + 1] - gstart[g]);
        grp0[i] = g;
        if (lh) lh[i] = h;
        if (unit) unit[i] = 1;
    }
}

inline int grid_for(Ctx &c, int64_t n) {
    int64_t b = ceil_div(n, DT);
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)c.num_sms * 16));
}

cudaError_t readback(Ctx &c, const void *dev, void *host, size_t bytes) {
    GJ_CUDA_TRY(cudaMemcpyAsync(c.pinned, dev, bytes, cudaMemcpyDeviceToHost, c.stream));
    GJ_CUDA_TRY(cudaStreamSynchronize(c.stream));
    memcpy(host, c.pinned, bytes);
    return cudaSuccess;
}

// The open subtrees beside preorder step j (see item_unit): simulate the DFS
// stack of the preorder walk.
std::vector<int> rest_at(const QueryState &q, int j) {
    std::vector<int> open(q.r[q.pre[0]].children);
    for (int step = 1; step <= j; step++) {
        int t = q.pre[step];
        // preorder: t is the top of the stack
        std::vector<int> next(q.r[t].children);
        next.insert(next.end(), open.begin() + 1, open.end());
        if (step == j) return std::vector<int>(open.begin() + 1, open.end());
        open.swap(next);
    }
    return {};
}

int child_index(const QRel &parent, int child_pos) {
    for (size_t i = 0; i < parent.children.size(); i++)
        if (parent.children[i] == child_pos) return (int)i;
    return -1;
}

// Frees a frontier when the scope ends, unless it was handed on.
struct FrontierHold {
    Ctx &c;
    Frontier &f;
    bool held = true;
    ~FrontierHold() {
        if (held) frontier_free(c, f);
    }
};

cudaError_t frontier_alloc(Ctx &c, Frontier &f, int64_t cap, int depth, bool keep_last,
                           bool need_w = true) {
    f.cap = cap;
    GJ_CUDA_TRY(dalloc(c, &f.F_dev, 1));
    GJ_CUDA_TRY(dalloc(c, &f.A, cap));
    if (need_w) GJ_CUDA_TRY(dalloc(c, &f.W, cap));
    f.grp.assign(depth, nullptr);
    for (int p = 0; p < depth; p++) GJ_CUDA_TRY(dalloc(c, &f.grp[p], cap));
    if (keep_last) {
        GJ_CUDA_TRY(dalloc(c, &f.lh, cap));
        GJ_CUDA_TRY(dalloc(c, &f.unit, cap));
    }
    return cudaSuccess;
}

// Frontier of path prefixes through preorder relations 0..depth-1 that
// overlap result rows [row0, row_end).  No host synchronisation: every
// frontier holds at most one item per row of the window, so arrays are
// sized by the window and item counts stay in device memory.
// keep_last: also fill lh and unit.  tm: the last level also writes the emit
// kernel's tile map (the block holding the first row of every emit tile).
struct TileMap {
    uint32_t *tile_first;   // [tiles + 1]
    int64_t tile_rows, tiles;
};

cudaError_t expand(QueryState &q, uint64_t row0, uint64_t row_end, int depth, bool keep_last,
                   Frontier &out, const TileMap *tm = nullptr) {
    Ctx &c = q.ctx();
    const QRel &root = q.r[q.pre[0]];
    const int64_t cap = (int64_t)(row_end - row0);
    const int pgrid = std::max(1, std::min<int>((int)ceil_div(cap, EXP_TILE), c.num_sms * 8));
    // every array is freed on the way out of an error
    Temps tmp(c);
    uint32_t *rr = nullptr;
    GJ_CUDA_TRY(tmp.alloc(&rr, 2));
    Frontier cur;
    FrontierHold hold_cur{c, cur};
    GJ_CUDA_TRY(frontier_alloc(c, cur, cap, 1, keep_last && depth == 1));
    k_root_range<<<1, 32, 0, c.stream>>>(root.loff, root.lw, root.L_dev, row0, row_end, rr,
                                        cur.F_dev); c.launches++;
    k_root_init<<<grid_for(c, cap), DT, 0, c.stream>>>(rr, cur.F_dev, root.lgid, root.loff,
                                                      root.F->gstart, cur.A, cur.W, cur.grp[0],
                                                      cur.lh, cur.unit); c.launches++;
    GJ_CUDA_TRY(cudaGetLastError());
    tmp.free(rr);
    for (int j = 1; j < depth; j++) {
        const int tpos = q.pre[j];
        const QRel &t = q.r[tpos];
        const QRel &par = q.r[t.parent];
        ExpandSpec s{};
        s.link = par.link[child_index(par, tpos)];
        s.parent_p = q.pos[t.parent];
        s.lseg_first = t.lseg_first;
        s.msg = t.msg;
        s.lgid = t.lgid;
        s.loff = t.loff;
        s.lw = t.lw;
        s.gstart = t.F->gstart;
        std::vector<int> rest = rest_at(q, j);
        s.nrest = (int)rest.size();
        for (int r = 0; r < s.nrest; r++) {
            const QRel &rc = q.r[rest[r]];
            const QRel &rp = q.r[rc.parent];
            s.rest_link[r] = rp.link[child_index(rp, rest[r])];
            s.rest_msg[r] = rc.msg;
            s.rest_parent_p[r] = q.pos[rc.parent];
        }
        s.depth = j;
        s.err = c.err;
        s.A = cur.A;
        s.W = cur.W;
        for (int p = 0; p < j; p++) s.grp[p] = cur.grp[p];
        Temps lt(c);   // this level's temporaries
        uint32_t *cnt = nullptr, *lo = nullptr, *excl = nullptr, *slot_first = nullptr;
        uint64_t *unit = nullptr;
        GJ_CUDA_TRY(lt.alloc(&cnt, cap));
        GJ_CUDA_TRY(lt.alloc(&lo, cap));
        GJ_CUDA_TRY(lt.alloc(&unit, cap));
        GJ_CUDA_TRY(lt.alloc(&excl, cap));
        GJ_CUDA_TRY(lt.alloc(&slot_first, ceil_div(cap, EXP_TILE) + 1));
        const bool last = (j == depth - 1);
        Frontier nxt;
        FrontierHold hold_nxt{c, nxt};
        // the last frontier's W (counts of the chosen groups) is not used
        GJ_CUDA_TRY(frontier_alloc(c, nxt, cap, j + 1, last && keep_last, !last));
        k_expand_count<<<grid_for(c, cap), DT, 0, c.stream>>>(s, cur.F_dev, row0, row_end, cnt, lo,
                                                            unit, c.err); c.launches++;
        GJ_CUDA_TRY(cudaGetLastError());
        GJ_CUDA_TRY(scan_u32_dev(c, cnt, nullptr, excl, cap, cur.F_dev, nxt.F_dev));
        ExpandOut o{};
        o.A = nxt.A;
        o.W = nxt.W;
        for (int p = 0; p <= j; p++) o.grp[p] = nxt.grp[p];
        o.lh = nxt.lh;
        o.unit = nxt.unit;
        if (last && tm) {
            o.tile_first = tm->tile_first;
            o.tile_rows = tm->tile_rows;
            o.tiles = tm->tiles;
            o.row0 = row0;
            o.n = (int64_t)(row_end - row0);
        }
        k_slot_first<<<grid_for(c, cap), DT, 0, c.stream>>>(excl, cnt, cur.F_dev, slot_first); c.launches++;
        k_expand_write<<<pgrid, DT, 0, c.stream>>>(s, cur.F_dev, excl, nxt.F_dev, slot_first, lo,
                                                   unit, o); c.launches++;
        GJ_CUDA_TRY(cudaGetLastError());
        frontier_free(c, cur);
        cur = nxt;               // held by hold_cur from here on
        hold_nxt.held = false;
    }
    out = cur;
    hold_cur.held = false;
    return cudaSuccess;
}

// ------------------------------------------------------------------ emission

constexpr int MAXV = 32;
constexpr int MAXP = 32;

struct EmitSpec {
    int k;                                // relations (query positions)
    int preidx[MAXR];                     // query position -> preorder index
    const uint32_t *gstart[MAXR];
    const uint32_t *perm[MAXR];
    uint32_t *rid_out[MAXR];
    int nv;
    const int32_t *vkey[MAXV];            // gkey row of the V column
    int vrel[MAXV];                       // query position owning it
    int32_t *vout[MAXV];
    int np;
    const void *pay[MAXP];
    int prel[MAXP];
    int pw[MAXP];
    void *pout[MAXP];
    const uint64_t *A;                    // block offsets
    const uint32_t *grp[MAXR];            // by preorder index
    uint32_t *err;
};

__global__ void __launch_bounds__(DT)
k_emit(EmitSpec e, const uint32_t *B_dev, uint64_t row0, int64_t n) {
    const int64_t B = *B_dev;
    __shared__ uint64_t s_A[EMIT_TILE + 1];
    __shared__ int64_t s_first;
    __shared__ int s_cnt;
    const int64_t r0 = (int64_t)blockIdx.x * EMIT_TILE;
    if (r0 >= n) return;
    const int64_t r1 = min(n, r0 + EMIT_TILE);
    if (threadIdx.x == 0) {
        int64_t a = 0, b = B;
        uint64_t x = row0 + (uint64_t)r0;
        while (a < b) { int64_t m = (a + b) >> 1; if (e.A[m] <= x) a = m + 1; else b = m; }
        int64_t first = a - 1;
        x = row0 + (uint64_t)(r1 - 1);
        a = first; b = B;
        while (a < b) { int64_t m = (a + b) >> 1; if (e.A[m] <= x) a = m + 1; else b = m; }
        s_first = first;
        int64_t cnt = a - first;
        if (first < 0 || cnt > EMIT_TILE) { raise_err(e.err, ERRF_BOUNDS); cnt = 0; }
        s_cnt = (int)cnt;
    }
    __syncthreads();
    const int64_t first = s_first;
    const int nb = s_cnt;
    if (nb == 0) return;
    for (int t = threadIdx.x; t < nb; t += DT) s_A[t] = e.A[first + t];
    __syncthreads();
    for (int64_t r = r0 + threadIdx.x; r < r1; r += DT) {
        const uint64_t row = row0 + (uint64_t)r;
        int a = 0, b = nb;
        while (a < b) { int m = (a + b) >> 1; if (s_A[m] <= row) a = m + 1; else b = m; }
        const int64_t blk = first + a - 1;
        uint64_t q = row - s_A[a - 1];
        uint32_t pos[MAXR];
        // mixed radix, relation k-1 fastest
        for (int j = e.k - 1; j >= 0; j--) {
            uint32_t g = e.grp[e.preidx[j]][blk];
            uint32_t base = e.gstart[j][g];
            uint32_t cnt = e.gstart[j][g + 1] - base;
            uint32_t d;
            if (q < 0x100000000ull) { uint32_t q32 = (uint32_t)q; d = q32 % cnt; q = q32 / cnt; }
            else { d = (uint32_t)(q % cnt); q /= cnt; }
            pos[j] = base + d;
        }
        for (int v = 0; v < e.nv; v++) {
            uint32_t g = e.grp[e.preidx[e.vrel[v]]][blk];
            e.vout[v][r] = e.vkey[v][g];
        }
        for (int p = 0; p < e.np; p++) {
            uint32_t at = pos[e.prel[p]];
            if (e.pw[p] == 8) ((uint64_t *)e.pout[p])[r] = ((const uint64_t *)e.pay[p])[at];
            else ((uint32_t *)e.pout[p])[r] = ((const uint32_t *)e.pay[p])[at];
        }
        for (int j = 0; j < e.k; j++)
            if (e.rid_out[j]) e.rid_out[j][r] = e.perm[j][pos[j]];
    }
}

// ------------------------------------------------------------------ levels

struct LevelSpec {
    const uint64_t *A;
    const uint32_t *lh;
    const uint64_t *unit;
    const uint32_t *lgid;
    const uint64_t *loff, *lw;
    const uint32_t *seg_id;       // NULL for the root
    const uint32_t *lseg_first;
    const uint32_t *L_dev;
    int nprefix;                  // new columns up to and including the level's
    bool last;                    // level's column is the relation's last new column
    const int32_t *pcol[MAX_KEYS];
    const int32_t *vcol;
};

__device__ __forceinline__ bool same_prefix(const LevelSpec &s, uint32_t g1, uint32_t g2) {
    for (int c = 0; c < s.nprefix; c++)
        if (s.pcol[c][g1] != s.pcol[c][g2]) return false;
    return true;
}

__global__ void k_level_flags(LevelSpec s, const uint32_t *F_dev, uint64_t row0, uint8_t *flag) {
    const int64_t F = *F_dev;
    for (int64_t i = (int64_t)blockIdx.x * DT + threadIdx.x; i < F; i += (int64_t)gridDim.x * DT) {
        uint8_t f = 0;
        if (s.A[i] >= row0) {
            uint32_t h = s.lh[i];
            uint32_t g = s.lgid[h];
            uint32_t a = s.seg_id ? s.lseg_first[s.seg_id[g]] : 0u;
            f = s.last || h == a || !same_prefix(s, s.lgid[h - 1], g);
        }
        flag[i] = f;
    }
}

__global__ void k_level_write(LevelSpec s, const uint32_t *F_dev, const uint8_t *flag,
                              const uint32_t *idx, int32_t *val, uint64_t *freq, uint64_t *off) {
    const int64_t F = *F_dev;
    for (int64_t i = (int64_t)blockIdx.x * DT + threadIdx.x; i < F; i += (int64_t)gridDim.x * DT) {
        if (!flag[i]) continue;
        uint32_t h = s.lh[i];
        uint32_t g = s.lgid[h];
        uint32_t he = h;
        if (!s.last) {
            uint32_t b = s.seg_id ? s.lseg_first[s.seg_id[g] + 1] : *s.L_dev;
            uint32_t a = h + 1;   // first live index after h with a different prefix
            while (a < b) {
                uint32_t m = a + ((b - a) >> 1);
                if (same_prefix(s, s.lgid[m], g)) a = m + 1; else b = m;
            }
            he = a - 1;
        }
        uint32_t o = idx[i];
        val[o] = s.vcol[g];
        freq[o] = s.unit[i] * (s.loff[he] + s.lw[he] - s.loff[h]);
        off[o] = s.A[i];
    }
}

}  // namespace

// The emit kernel's description of a query's output: for every relation
// (query position j) its factor, its block groups grp[j] and its output
// columns (key columns of V, then payloads).  False if the layout exceeds
// the kernel's limits.
bool make_emit_spec(QueryState &q, void *const *out_cols, uint32_t *const *rowid_cols,
                    const uint32_t *const *grp, const uint64_t *A, Emit4Spec &s) {
    s = Emit4Spec{};
    if (q.k > EMIT_MAXR || (int)q.var_rel.size() > EMIT_MAXV || (int)q.col_rel.size() > EMIT_MAXP)
        return false;
    int nc = 0;
    bool vec = true;
    const int nv = (int)q.var_rel.size();
    for (int j = 0; j < q.k; j++) {
        s.gstart[j] = q.r[j].F->gstart;
        s.perm[j] = q.r[j].F->perm;
        s.rid_out[j] = rowid_cols ? rowid_cols[j] : nullptr;
        s.grp[j] = grp[j];
        s.col_off[j] = nc;
        for (int v = 0; v < nv; v++) {
            if (q.var_rel[v] != j) continue;
            s.src[nc] = q.r[j].F->gkey + (int64_t)q.var_col[v] * q.r[j].F->G;
            s.dst[nc] = out_cols[v];
            s.kind[nc] = 0;
            nc++;
        }
        for (size_t p = 0; p < q.col_rel.size(); p++) {
            if (q.col_rel[p] != j) continue;
            s.src[nc] = q.r[j].F->pay[q.col_pay[p]];
            s.dst[nc] = out_cols[nv + p];
            s.kind[nc] = q.r[j].R->pw[q.col_pay[p]] == 8 ? 2 : 1;
            nc++;
        }
    }
    s.col_off[q.k] = nc;
    // 32-byte vector stores need 32-byte aligned columns
    for (int i = 0; i < nc; i++) vec &= ((uintptr_t)s.dst[i] & 31) == 0;
    s.vec = vec;
    s.A = A;
    s.err = q.ctx().err;
    return true;
}

gj_status tri_desummarize(QueryState &q, uint64_t row0, uint64_t nrows, void *const *out_cols,
                          uint32_t *const *rowid_cols, uint64_t *n_out);

gj_status cyc_desummarize(QueryState &q, uint64_t row0, uint64_t nrows, void *const *out_cols,
                          uint32_t *const *rowid_cols, uint64_t *n_out);

gj_status desummarize(QueryState &q, uint64_t row0, uint64_t nrows, void *const *out_cols,
                      uint32_t *const *rowid_cols, uint64_t *n_out) {
    if (q.tri) return tri_desummarize(q, row0, nrows, out_cols, rowid_cols, n_out);
    if (q.cyc) return cyc_desummarize(q, row0, nrows, out_cols, rowid_cols, n_out);
    Ctx &c = q.ctx();
    *n_out = 0;
    if (!q.summarized) return GJ_ERR_STATE;
    if (q.overflow) return GJ_ERR_OVERFLOW;
    if (row0 >= q.total || nrows == 0) return GJ_OK;
    uint64_t n = std::min<uint64_t>(nrows, q.total - row0);
    if (n > 0x7fffffffull) return GJ_ERR_INVALID;
    if ((int)q.var_rel.size() > MAXV || (int)q.col_rel.size() > MAXP) return GJ_ERR_INVALID;
    if (!out_cols) return GJ_ERR_INVALID;
    Frontier f;
    if (c.prof) cudaEventRecord(c.event(true), c.stream);
    // with two or more relations the last expansion level writes the emit
    // kernel's tile map itself
    TileMap tm{};
    if (q.k >= 2 && q.k <= 8) {
        tm.tile_rows = (int64_t)EMIT_DT * c.emit_rpt;
        tm.tiles = ceil_div((int64_t)n, tm.tile_rows);
        if (dalloc(c, &tm.tile_first, tm.tiles + 1) != cudaSuccess) return GJ_ERR_OOM;
    }
    cudaError_t e = expand(q, row0, row0 + n, q.k, false, f, tm.tile_first ? &tm : nullptr);
    if (c.prof) cudaEventRecord(c.event(true), c.stream);
    if (e != cudaSuccess) {
        dfree(c, tm.tile_first);
        return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
    }
    uint64_t width = 0;
    for (int v = 0; v < (int)q.var_rel.size(); v++) width += 4;
    for (size_t p = 0; p < q.col_rel.size(); p++) width += q.r[q.col_rel[p]].R->pw[q.col_pay[p]];
    if (q.k > 8 && c.prof) cudaEventRecord(c.event(), c.stream);
    if (q.k <= 8) {
        Emit4Spec s{};
        std::vector<const uint32_t *> grp(q.k);
        for (int j = 0; j < q.k; j++) grp[j] = f.grp[q.pos[j]];
        make_emit_spec(q, out_cols, rowid_cols, grp.data(), f.A, s);
        e = launch_emit(c, q.k, s, f.F_dev, row0, (int64_t)n, tm.tile_first);
    } else {
        EmitSpec s{};
        s.k = q.k;
        for (int j = 0; j < q.k; j++) {
            s.preidx[j] = q.pos[j];
            s.gstart[j] = q.r[j].F->gstart;
            s.perm[j] = q.r[j].F->perm;
            s.rid_out[j] = rowid_cols ? rowid_cols[j] : nullptr;
            s.grp[j] = f.grp[j];
        }
        s.nv = (int)q.var_rel.size();
        for (int v = 0; v < s.nv; v++) {
            const QRel &t = q.r[q.var_rel[v]];
            s.vkey[v] = t.F->gkey + (int64_t)q.var_col[v] * t.F->G;
            s.vrel[v] = q.var_rel[v];
            s.vout[v] = (int32_t *)out_cols[v];
        }
        s.np = (int)q.col_rel.size();
        for (int p = 0; p < s.np; p++) {
            const QRel &t = q.r[q.col_rel[p]];
            s.pay[p] = t.F->pay[q.col_pay[p]];
            s.prel[p] = q.col_rel[p];
            s.pw[p] = t.R->pw[q.col_pay[p]];
            s.pout[p] = out_cols[s.nv + p];
        }
        s.A = f.A;
        s.err = c.err;
        k_emit<<<(unsigned)ceil_div((int64_t)n, EMIT_TILE), DT, 0, c.stream>>>(s, f.F_dev, row0, (int64_t)n); c.launches++;
        e = cudaGetLastError();
    }
    if (c.prof) {
        cudaEventRecord(c.event(), c.stream);
        c.emit_launches++;
        c.emit_rows += n;
        c.emit_bytes += n * width;
    }
    frontier_free(c, f);
    dfree(c, tm.tile_first);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
    gj_status st = check_device_error(c);
    if (st != GJ_OK) return st;
    *n_out = n;
    return GJ_OK;
}

gj_status level_runs(QueryState &q, int level, uint64_t row0, uint64_t nrows, int32_t *val,
                     uint64_t *freq, uint64_t *off, uint64_t cap, uint64_t *n_out) {
    Ctx &c = q.ctx();
    *n_out = 0;
    if (q.tri || q.cyc) return GJ_ERR_INVALID;   // a cyclic join's summary is its block list
    if (!q.summarized) return GJ_ERR_STATE;
    if (q.overflow) return GJ_ERR_OVERFLOW;
    if (level < 0 || level >= (int)q.var_rel.size()) return GJ_ERR_INVALID;
    if (row0 >= q.total || nrows == 0) return GJ_OK;
    uint64_t n = std::min<uint64_t>(nrows, q.total - row0);
    if (n > 0x7fffffffull) return GJ_ERR_INVALID;
    const int tpos = q.var_rel[level];
    const QRel &t = q.r[tpos];
    const int j = q.pos[tpos];
    Frontier f;
    cudaError_t e = expand(q, row0, row0 + n, j + 1, true, f);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
    LevelSpec s{};
    s.A = f.A;
    s.lh = f.lh;
    s.unit = f.unit;
    s.lgid = t.lgid;
    s.loff = t.loff;
    s.lw = t.lw;
    s.seg_id = t.parent >= 0 ? t.seg_id : nullptr;
    s.lseg_first = t.lseg_first;
    s.L_dev = t.L_dev;
    int m = -1;
    for (size_t i = 0; i < t.new_cols.size(); i++)
        if (t.new_cols[i] == q.var_col[level]) m = (int)i;
    s.nprefix = m + 1;
    s.last = (m == (int)t.new_cols.size() - 1);
    for (int i = 0; i <= m; i++) s.pcol[i] = t.F->gkey + (int64_t)t.new_cols[i] * t.F->G;
    s.vcol = t.F->gkey + (int64_t)q.var_col[level] * t.F->G;
    uint8_t *flag = nullptr;
    uint32_t *idx = nullptr, *tot = nullptr;
    gj_status st = GJ_OK;
    uint32_t R = 0;
    if ((e = dalloc(c, &flag, f.cap)) != cudaSuccess) goto fail;
    if ((e = dalloc(c, &idx, f.cap)) != cudaSuccess) goto fail;
    if ((e = dalloc(c, &tot, 1)) != cudaSuccess) goto fail;
    k_level_flags<<<grid_for(c, f.cap), DT, 0, c.stream>>>(s, f.F_dev, row0, flag); c.launches++;
    if ((e = scan_u32_dev(c, nullptr, flag, idx, f.cap, f.F_dev, tot)) != cudaSuccess) goto fail;
    if ((e = readback(c, tot, &R, 4)) != cudaSuccess) goto fail;
    *n_out = R;
    if (R > cap) { st = GJ_ERR_CAPACITY; goto done; }
    k_level_write<<<grid_for(c, f.cap), DT, 0, c.stream>>>(s, f.F_dev, flag, idx, val, freq, off); c.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
    st = check_device_error(c);
    goto done;
fail:
    st = e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
done:
    dfree(c, flag);
    dfree(c, idx);
    dfree(c, tot);
    frontier_free(c, f);
    return st;
}

}  // namespace gj
