// gj_cycle.cu -- the cyclic 3-way join R(A,B) |><| S(B,C) |><| T(C,A).
//
// A cycle has no join tree.  The paper builds a junction tree instead
// (Section 2.3: min-fill-in triangulation of the moral graph) and computes
// the potential of every cluster as the join of the potentials of its
// relations (Algorithm 1).  For three relations pairwise sharing one
// attribute the triangulation leaves one cluster {A, B, C}, so the summary
// is that cluster's potential: every triple of groups (g_R, g_S, g_T) with
// g_R = (a, b), g_S = (b, c), g_T = (c, a), holding cnt_R * cnt_S * cnt_T
// result rows.  These triples are exactly the blocks the desummarise emit
// kernel expands (rows of a block ordered by r_R, r_S, r_T, the last
// fastest), so the cyclic query reuses it unchanged.
//
// The cluster potential is built from the sorted factors, in result order:
//   1. per R group (a, b) (R's factor order), the S groups with key b form
//      one contiguous segment of S's factor, ordered by (b, c): its wedges;
//   2. an exclusive scan numbers the wedges; one thread per wedge looks its
//      closing edge (c, a) up in T's factor, ordered by (c, a);
//   3. a scan over the hits numbers the blocks; each writes its three groups
//      and its row count (saturating product); a saturating scan gives the
//      blocks' first rows and |Q|.
// Wedges are walked in R-group order and, inside, in c order, so blocks come
// out ordered by (V_0, V_1, c) with V the root's columns then C.
#include <string.h>

#include <algorithm>

#include "gj_emit.cuh"

namespace gj {

gj_status check_device_error(Ctx &c);
bool make_emit_spec(QueryState &q, void *const *out_cols, uint32_t *const *rowid_cols,
                    const uint32_t *const *grp, const uint64_t *A, Emit4Spec &s);

namespace {

constexpr int CT = 256;

struct TriSpec {
    const int32_t *a0, *b0;         // R's groups: the attribute shared with T, with S
    const uint32_t *gs0;
    int64_t G0;
    const int32_t *b1, *c1;         // S's groups, ordered by (b, c)
    const uint32_t *gs1;
    int64_t G1;
    const int32_t *c2, *a2;         // T's groups, ordered by (c, a)
    const uint32_t *gs2;
    int64_t G2;
};

inline int grid_for(Ctx &c, int64_t n) {
    int64_t b = ceil_div(n, CT);
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)c.num_sms * 16));
}

// first index in [lo, hi) whose key exceeds x (keys ascending)
__device__ __forceinline__ uint32_t upper_i32(const int32_t *k, uint32_t lo, uint32_t hi, int32_t x) {
    while (lo < hi) {
        uint32_t m = lo + ((hi - lo) >> 1);
        if (k[m] <= x) lo = m + 1; else hi = m;
    }
    return lo;
}
__device__ __forceinline__ uint32_t lower_i32(const int32_t *k, uint32_t lo, uint32_t hi, int32_t x) {
    while (lo < hi) {
        uint32_t m = lo + ((hi - lo) >> 1);
        if (k[m] < x) lo = m + 1; else hi = m;
    }
    return lo;
}

// S's segment of every R group, and the exact number of wedges (64-bit)
__global__ void k_tri_deg(TriSpec s, uint32_t *lo, uint32_t *deg, unsigned long long *wsum) {
    unsigned long long mine = 0;
    for (int64_t i = (int64_t)blockIdx.x * CT + threadIdx.x; i < s.G0; i += (int64_t)gridDim.x * CT) {
        const int32_t b = s.b0[i];
        const uint32_t l = lower_i32(s.b1, 0, (uint32_t)s.G1, b);
        const uint32_t h = upper_i32(s.b1, l, (uint32_t)s.G1, b);
        lo[i] = l;
        deg[i] = h - l;
        mine += h - l;
    }
    for (int d = 16; d; d >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, d);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(wsum, mine);
}

// the T group holding (c, a), or NONE
__device__ __forceinline__ uint32_t find_ca(const TriSpec &s, int32_t c, int32_t a) {
    uint32_t l = lower_i32(s.c2, 0, (uint32_t)s.G2, c);
    const uint32_t h = upper_i32(s.c2, l, (uint32_t)s.G2, c);
    l = lower_i32(s.a2, l, h, a);
    return (l < h && s.a2[l] == a) ? l : NONE;
}

// wedge w belongs to the last R group i with woff[i] <= w
__device__ __forceinline__ uint32_t wedge_owner(const uint32_t *woff, int64_t G0, uint64_t w) {
    uint32_t lo = 0, hi = (uint32_t)G0;
    while (lo < hi) {
        uint32_t m = lo + ((hi - lo) >> 1);
        if ((uint64_t)woff[m] <= w) lo = m + 1; else hi = m;
    }
    return lo - 1;
}

__global__ void k_tri_check(TriSpec s, const uint32_t *__restrict__ lo, const uint32_t *__restrict__ woff,
                            uint64_t nw, uint32_t *t_of, uint8_t *hit, uint32_t *err) {
    for (uint64_t w = (uint64_t)blockIdx.x * CT + threadIdx.x; w < nw; w += (uint64_t)gridDim.x * CT) {
        const uint32_t i = wedge_owner(woff, s.G0, w);
        const uint32_t j = lo[i] + (uint32_t)(w - woff[i]);
        uint32_t t = NONE;
        if (i < s.G0 && j < s.G1) t = find_ca(s, s.c1[j], s.a0[i]);
        else raise_err(err, ERRF_BOUNDS);
        t_of[w] = t;
        hit[w] = t != NONE;
    }
}

__global__ void k_tri_write(TriSpec s, const uint32_t *__restrict__ lo, const uint32_t *__restrict__ woff,
                            uint64_t nw, const uint32_t *__restrict__ t_of, const uint8_t *__restrict__ hit,
                            const uint32_t *__restrict__ bidx, uint32_t *g0, uint32_t *g1, uint32_t *g2,
                            uint64_t *W) {
    for (uint64_t w = (uint64_t)blockIdx.x * CT + threadIdx.x; w < nw; w += (uint64_t)gridDim.x * CT) {
        if (!hit[w]) continue;
        const uint32_t i = wedge_owner(woff, s.G0, w);
        const uint32_t j = lo[i] + (uint32_t)(w - woff[i]);
        const uint32_t t = t_of[w];
        const uint32_t b = bidx[w];
        g0[b] = i;
        g1[b] = j;
        g2[b] = t;
        const uint64_t c0 = s.gs0[i + 1] - s.gs0[i], c1 = s.gs1[j + 1] - s.gs1[j],
                       c2 = s.gs2[t + 1] - s.gs2[t];
        W[b] = sat_mul(sat_mul(c0, c1), c2);
    }
}

// blocks overlapping result rows [row0, row_end): out = {first, count}
__global__ void k_tri_window(const uint64_t *A, uint64_t B, uint64_t row0, uint64_t row_end,
                             uint32_t *out) {
    auto last_le = [&](uint64_t x) {   // last block whose first row <= x
        uint64_t lo = 0, hi = B;
        while (lo < hi) {
            uint64_t m = (lo + hi) >> 1;
            if (A[m] <= x) lo = m + 1; else hi = m;
        }
        return lo - 1;
    };
    const uint64_t f = last_le(row0), l = last_le(row_end - 1);
    out[0] = (uint32_t)f;
    out[1] = (uint32_t)(l - f + 1);
}

cudaError_t readback(Ctx &c, const void *dev, void *host, size_t bytes) {
    GJ_CUDA_TRY(cudaMemcpyAsync(c.pinned, dev, bytes, cudaMemcpyDeviceToHost, c.stream));
    GJ_CUDA_TRY(cudaStreamSynchronize(c.stream));
    memcpy(host, c.pinned, bytes);
    return cudaSuccess;
}

TriSpec tri_spec(QueryState &q) {
    TriSpec s{};
    const Factor &F0 = *q.r[0].F, &F1 = *q.r[1].F, &F2 = *q.r[2].F;
    s.a0 = F0.gkey + (int64_t)q.tri_col[0][0] * F0.G;
    s.b0 = F0.gkey + (int64_t)q.tri_col[0][1] * F0.G;
    s.gs0 = F0.gstart;
    s.G0 = F0.G;
    s.b1 = F1.gkey + (int64_t)q.tri_col[1][0] * F1.G;
    s.c1 = F1.gkey + (int64_t)q.tri_col[1][1] * F1.G;
    s.gs1 = F1.gstart;
    s.G1 = F1.G;
    s.c2 = F2.gkey + (int64_t)q.tri_col[2][0] * F2.G;
    s.a2 = F2.gkey + (int64_t)q.tri_col[2][1] * F2.G;
    s.gs2 = F2.gstart;
    s.G2 = F2.G;
    return s;
}

}  // namespace

void tri_free(Ctx &c, QueryState &q) {
    dfree(c, q.blk_A);
    for (auto &g : q.blk_grp) dfree(c, g);
    q.nblocks = 0;
}

gj_status tri_summarize(QueryState &q, uint64_t *total_out) {
    Ctx &c = q.ctx();
    tri_free(c, q);
    q.summarized = false;
    const TriSpec s = tri_spec(q);
    uint32_t *lo = nullptr, *deg = nullptr, *woff = nullptr, *cnt = nullptr, *t_of = nullptr,
             *bidx = nullptr;
    uint8_t *hit = nullptr;
    uint64_t *W = nullptr, *total_dev = nullptr;
    unsigned long long *wsum = nullptr;
    unsigned long long nw_exact = 0;
    uint32_t nw32 = 0, nb32 = 0;
    uint64_t total = 0;
    gj_status st = GJ_OK;
    cudaError_t e = cudaSuccess;
#define TRY(x)                                                 \
    do {                                                       \
        e = (x);                                               \
        if (e != cudaSuccess) {                                \
            note_cuda_error(e, __FILE__, __LINE__);            \
            goto fail;                                         \
        }                                                      \
    } while (0)
    TRY(dalloc(c, &cnt, 2));
    TRY(dalloc(c, &total_dev, 1));
    if (s.G0 > 0 && s.G1 > 0 && s.G2 > 0) {
        // 1. wedges per R group
        TRY(dalloc(c, &lo, s.G0));
        TRY(dalloc(c, &deg, s.G0));
        TRY(dalloc(c, &woff, s.G0));
        TRY(dalloc(c, &wsum, 1));
        TRY(cudaMemsetAsync(wsum, 0, sizeof(unsigned long long), c.stream));
        k_tri_deg<<<grid_for(c, s.G0), CT, 0, c.stream>>>(s, lo, deg, wsum); c.launches++;
        TRY(cudaGetLastError());
        TRY(readback(c, wsum, &nw_exact, 8));
        // wedges are numbered in 32 bits
        if (nw_exact > 0x7fffffffull) { st = GJ_ERR_CAPACITY; goto done; }
        TRY(scan_u32(c, deg, nullptr, woff, s.G0, cnt));
        TRY(readback(c, cnt, &nw32, 4));
        uint64_t nw = nw32;
        if (nw != nw_exact) { st = GJ_ERR_CUDA; goto done; }   // cannot happen
        if (nw > 0) {
            // 2. closing edges, 3. blocks
            TRY(dalloc(c, &t_of, nw));
            TRY(dalloc(c, &hit, nw));
            TRY(dalloc(c, &bidx, nw));
            k_tri_check<<<grid_for(c, (int64_t)nw), CT, 0, c.stream>>>(s, lo, woff, nw, t_of, hit, c.err); c.launches++;
            TRY(cudaGetLastError());
            TRY(scan_u32(c, nullptr, hit, bidx, (int64_t)nw, cnt + 1));
            TRY(readback(c, cnt + 1, &nb32, 4));
            if (nb32 > 0) {
                for (auto &g : q.blk_grp) TRY(dalloc(c, &g, nb32));
                TRY(dalloc(c, &W, nb32));
                TRY(dalloc(c, &q.blk_A, nb32));
                k_tri_write<<<grid_for(c, (int64_t)nw), CT, 0, c.stream>>>(
                    s, lo, woff, nw, t_of, hit, bidx, q.blk_grp[0], q.blk_grp[1], q.blk_grp[2], W); c.launches++;
                TRY(cudaGetLastError());
                TRY(scan_u64_sat(c, W, nullptr, q.blk_A, nb32, total_dev, nullptr, nullptr));
                TRY(readback(c, total_dev, &total, 8));
            }
        }
    }
    st = check_device_error(c);
    if (st != GJ_OK) goto done;
    q.nblocks = nb32;
    q.total = total;
    q.overflow = total == SAT;
    q.summarized = true;
    if (total_out) *total_out = total;
    st = q.overflow ? GJ_ERR_OVERFLOW : GJ_OK;
    goto done;
fail:
    st = e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
done:
#undef TRY
    if (!q.summarized) tri_free(c, q);
    dfree(c, lo);
    dfree(c, deg);
    dfree(c, woff);
    dfree(c, cnt);
    dfree(c, t_of);
    dfree(c, hit);
    dfree(c, bidx);
    dfree(c, W);
    dfree(c, total_dev);
    dfree(c, wsum);
    return st;
}

gj_status tri_desummarize(QueryState &q, uint64_t row0, uint64_t nrows, void *const *out_cols,
                          uint32_t *const *rowid_cols, uint64_t *n_out) {
    Ctx &c = q.ctx();
    *n_out = 0;
    if (!q.summarized) return GJ_ERR_STATE;
    if (q.overflow) return GJ_ERR_OVERFLOW;
    if (row0 >= q.total || nrows == 0) return GJ_OK;
    const uint64_t n = std::min<uint64_t>(nrows, q.total - row0);
    if (n > 0x7fffffffull || !out_cols) return GJ_ERR_INVALID;
    uint32_t *win = nullptr;
    uint32_t w[2] = {0, 0};
    if (dalloc(c, &win, 2) != cudaSuccess) return GJ_ERR_OOM;
    k_tri_window<<<1, 1, 0, c.stream>>>(q.blk_A, q.nblocks, row0, row0 + n, win); c.launches++;
    if (cudaGetLastError() != cudaSuccess || readback(c, win, w, 8) != cudaSuccess) {
        dfree(c, win);
        return GJ_ERR_CUDA;
    }
    gj_status st = GJ_OK;
    if ((uint64_t)w[0] + w[1] > q.nblocks || w[1] == 0) {
        st = GJ_ERR_CUDA;   // cannot happen: the window lies inside |Q|
    } else {
        const uint32_t *grp[3] = {q.blk_grp[0] + w[0], q.blk_grp[1] + w[0], q.blk_grp[2] + w[0]};
        Emit4Spec s{};
        if (!make_emit_spec(q, out_cols, rowid_cols, grp, q.blk_A + w[0], s)) {
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
            st = e != cudaSuccess ? GJ_ERR_CUDA : check_device_error(c);
        }
    }
    dfree(c, win);
    if (st == GJ_OK) *n_out = n;
    return st;
}

}  // namespace gj
