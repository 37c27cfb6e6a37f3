// gj_summary.cu -- the sum-product passes that summarise the join.
//
// Upward (Algorithm 2 on a tree, Eqs. 6-10).  The join tree is processed
// leaves to root.  For a relation t with groups g (distinct key tuples,
// count cnt[g]) and children c:
//
//     w[g]     = cnt[g] (x) prod_c msg_c[ link_c(g) ]         (product, line 6)
//     msg_t[s] = (+)_{g : sep(g) = s} w[g]                   (sum-out, line 9)
//
// where link_c(g) is the segment of c whose separator values equal g's, and
// a missing segment contributes 0 (a dead branch, pruned as the paper drops
// entries below 1).  cnt[g] is the paper's bucket, the product over the
// children is its fac.  At the root, (+)_g w[g] = |Q| (the root marginal
// sums to the join size, Section 3.3).  (+) and (x) are the saturating
// semiring operations of gj_internal.cuh.
//
// Offsets (Algorithms 3-4).  The root's groups in key order each own the
// result rows [off[g], off[g] + w[g]) with off the exclusive scan of w.  A
// non-root group's rel_off is the exclusive scan of w within its separator
// segment: inside a parent path that owns `unit` rows per child way, group
// g owns rows [unit * rel_off[g], unit * (rel_off[g] + w[g])) -- the
// bucket_new = p_bucket * bucket product of Algorithm 4.
//
// Downward.  down_c[s] counts the completions of the rest of the tree given
// c's separator value s:  (+) over parent groups g linking to s of
// down_t(g) (x) cnt[g] (x) prod_{c' != c} msg_c'.  mult[g] = w[g] (x) down(g)
// is the number of result tuples using group g, i.e. the marginal of g's key
// tuple over the join result (Section 1.2, "Why PGMs").
#include <algorithm>

#include "gj_state.cuh"

namespace gj {

void note_cuda_error(cudaError_t e, const char *file, int line);

namespace {

constexpr int ST = 256;
constexpr int64_t DENSE_MAX = 1ll << 26;   // largest dense link table (entries)

struct KeyCols {
    int ncol;
    const int32_t *col[MAX_KEYS];
};

struct ChildSet {
    int n;
    const uint32_t *link[MAX_REL];
    const uint64_t *msg[MAX_REL];
    unsigned long long *lo[MAX_REL];
    unsigned int *carry[MAX_REL];
};

inline int grid_for(Ctx &c, int64_t n) {
    int64_t b = ceil_div(n, ST);
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)c.num_sms * 16));
}

#define GRID_LOOP(i, n) \
    for (int64_t i = (int64_t)blockIdx.x * ST + threadIdx.x; i < (n); i += (int64_t)gridDim.x * ST)

__global__ void k_seg_heads(KeyCols sep, int64_t G, uint8_t *heads) {
    GRID_LOOP(g, G) {
        uint8_t h = (g == 0);
        if (!h)
            for (int c = 0; c < sep.ncol; c++)
                if (sep.col[c][g] != sep.col[c][g - 1]) { h = 1; break; }
        heads[g] = h;
    }
}

__global__ void k_seg_finalize(const uint8_t *heads, const uint32_t *excl, int64_t G,
                               const uint32_t *S_dev, uint32_t *seg_id, uint32_t *seg_first) {
    GRID_LOOP(g, G) {
        uint32_t s = excl[g] + heads[g] - 1u;
        seg_id[g] = s;
        if (heads[g]) seg_first[s] = (uint32_t)g;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) seg_first[*S_dev] = (uint32_t)G;
}

__global__ void k_fill_u32(uint32_t *p, int64_t n, uint32_t v) {
    GRID_LOOP(i, n) p[i] = v;
}

__global__ void k_dense_fill(const int32_t *child_key, const uint32_t *seg_first,
                             const uint32_t *S_dev, int32_t mn, uint32_t *dense) {
    const int64_t S = *S_dev;
    GRID_LOOP(s, S) dense[(uint32_t)child_key[seg_first[s]] - (uint32_t)mn] = (uint32_t)s;
}

__global__ void k_link_dense(const int32_t *parent_key, int64_t Gp, int32_t mn, uint64_t range,
                             const uint32_t *dense, uint32_t *link) {
    GRID_LOOP(g, Gp) {
        uint32_t d = (uint32_t)parent_key[g] - (uint32_t)mn;
        link[g] = (uint64_t)d < range ? dense[d] : NONE;
    }
}

__global__ void k_link_search(KeyCols pk, int64_t Gp, KeyCols ck, const uint32_t *seg_first,
                              const uint32_t *S_dev, uint32_t *link) {
    const int64_t S = *S_dev;
    GRID_LOOP(g, Gp) {
        int32_t want[MAX_KEYS];
        for (int c = 0; c < pk.ncol; c++) want[c] = pk.col[c][g];
        int64_t lo = 0, hi = S;   // first segment whose key >= want
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            uint32_t f = seg_first[mid];
            int cmp = 0;
            for (int c = 0; c < ck.ncol && cmp == 0; c++) {
                int32_t v = ck.col[c][f];
                cmp = v < want[c] ? -1 : (v > want[c] ? 1 : 0);
            }
            if (cmp < 0) lo = mid + 1; else hi = mid;
        }
        uint32_t r = NONE;
        if (lo < S) {
            uint32_t f = seg_first[lo];
            bool eq = true;
            for (int c = 0; c < ck.ncol; c++) eq &= ck.col[c][f] == want[c];
            if (eq) r = (uint32_t)lo;
        }
        link[g] = r;
    }
}

__global__ void k_weights(const uint32_t *gstart, int64_t G, ChildSet ch, uint64_t *w) {
    GRID_LOOP(g, G) {
        uint64_t v = (uint64_t)(gstart[g + 1] - gstart[g]);
        for (int i = 0; i < ch.n; i++) {
            uint32_t s = ch.link[i][g];
            v = sat_mul(v, s == NONE ? 0ull : ch.msg[i][s]);
        }
        w[g] = v;
    }
}

// contributions of t's groups to every child's down message
__global__ void k_down_contrib(const uint32_t *gstart, int64_t G, const uint64_t *t_down,
                               const uint32_t *t_seg, ChildSet ch) {
    GRID_LOOP(g, G) {
        uint64_t base = (uint64_t)(gstart[g + 1] - gstart[g]);
        if (t_down) base = sat_mul(base, t_down[t_seg[g]]);
        if (base == 0) continue;
        for (int i = 0; i < ch.n; i++) {
            uint32_t s = ch.link[i][g];
            if (s == NONE) continue;
            uint64_t x = base;
            for (int j = 0; j < ch.n && x; j++) {
                if (j == i) continue;
                uint32_t sj = ch.link[j][g];
                x = sat_mul(x, sj == NONE ? 0ull : ch.msg[j][sj]);
            }
            if (x == 0) continue;
            // exact sum modulo 2^64 plus a wrap counter: saturates iff the
            // true sum is >= 2^64 - 1, with native 64-bit atomics
            if (x == SAT) { atomicOr(&ch.carry[i][s], 1u); continue; }
            unsigned long long old = atomicAdd(&ch.lo[i][s], (unsigned long long)x);
            if (old + x < old) atomicOr(&ch.carry[i][s], 1u);
        }
    }
}

__global__ void k_down_finalize(const unsigned long long *lo, const unsigned int *carry,
                                const uint32_t *S_dev, uint64_t *down) {
    const int64_t S = *S_dev;
    GRID_LOOP(s, S) down[s] = (carry[s] || lo[s] == SAT) ? SAT : (uint64_t)lo[s];
}

__global__ void k_mult(const uint64_t *w, const uint64_t *t_down, const uint32_t *t_seg, int64_t G,
                       uint64_t *mult) {
    GRID_LOOP(g, G) mult[g] = t_down ? sat_mul(w[g], t_down[t_seg[g]]) : w[g];
}

__global__ void k_nonzero(const uint64_t *w, int64_t G, uint8_t *f) {
    GRID_LOOP(g, G) f[g] = w[g] != 0;
}

__global__ void k_live_compact(const uint8_t *f, const uint32_t *lidx, const uint64_t *w,
                               const uint64_t *off, int64_t G, uint32_t *lgid, uint64_t *loff,
                               uint64_t *lw) {
    GRID_LOOP(g, G) {
        if (!f[g]) continue;
        uint32_t h = lidx[g];
        lgid[h] = (uint32_t)g;
        loff[h] = off[g];
        lw[h] = w[g];
    }
}

__global__ void k_live_segs(const uint32_t *seg_first, const uint32_t *lidx,
                            const uint32_t *S_dev, const uint32_t *L_dev, uint32_t *lseg_first) {
    const int64_t S = *S_dev;
    GRID_LOOP(s, S) lseg_first[s] = lidx[seg_first[s]];
    if (blockIdx.x == 0 && threadIdx.x == 0) lseg_first[S] = *L_dev;
}

inline KeyCols key_cols(const QRel &q, const std::vector<int> &cols) {
    KeyCols k{};
    k.ncol = (int)cols.size();
    for (int i = 0; i < k.ncol; i++) k.col[i] = q.F->gkey + (int64_t)cols[i] * q.F->G;
    return k;
}

cudaError_t build_segments(Ctx &c, QRel &t) {
    const int64_t G = t.F->G;
    GJ_CUDA_TRY(dalloc(c, &t.seg_id, G));
    GJ_CUDA_TRY(dalloc(c, &t.seg_first, G + 1));
    GJ_CUDA_TRY(dalloc(c, &t.S_dev, 1));
    uint8_t *heads = nullptr;
    uint32_t *excl = nullptr;
    GJ_CUDA_TRY(dalloc(c, &heads, G));
    GJ_CUDA_TRY(dalloc(c, &excl, G));
    k_seg_heads<<<grid_for(c, G), ST, 0, c.stream>>>(key_cols(t, t.sep_cols), G, heads); c.launches++;
    GJ_CUDA_TRY(scan_u32(c, nullptr, heads, excl, G, t.S_dev));
    k_seg_finalize<<<grid_for(c, G), ST, 0, c.stream>>>(heads, excl, G, t.S_dev, t.seg_id, t.seg_first); c.launches++;
    GJ_CUDA_TRY(cudaGetLastError());
    dfree(c, heads);
    dfree(c, excl);
    return cudaSuccess;
}

// link[g] for every group g of parent t: segment of child ch with equal
// separator values, or NONE
cudaError_t build_link(Ctx &c, QRel &t, QRel &ch, uint32_t **link_out) {
    const int64_t Gp = t.F->G;
    uint32_t *link = nullptr;
    GJ_CUDA_TRY(dalloc(c, &link, Gp));
    *link_out = link;
    if (Gp == 0) return cudaSuccess;
    if (ch.F->G == 0) {
        k_fill_u32<<<grid_for(c, Gp), ST, 0, c.stream>>>(link, Gp, NONE); c.launches++;
        return cudaGetLastError();
    }
    if (ch.sep_cols.size() == 1) {
        int col = ch.sep_cols[0];
        int64_t range = (int64_t)ch.R->kmax[col] - (int64_t)ch.R->kmin[col] + 1;
        if (range <= DENSE_MAX && range <= 4 * (ch.F->G + Gp) + 4096) {
            uint32_t *dense = nullptr;
            GJ_CUDA_TRY(dalloc(c, &dense, range));
            GJ_CUDA_TRY(cudaMemsetAsync(dense, 0xFF, sizeof(uint32_t) * range, c.stream));
            k_dense_fill<<<grid_for(c, ch.F->G), ST, 0, c.stream>>>(
                ch.F->gkey + (int64_t)col * ch.F->G, ch.seg_first, ch.S_dev, ch.R->kmin[col], dense); c.launches++;
            k_link_dense<<<grid_for(c, Gp), ST, 0, c.stream>>>(
                t.F->gkey + (int64_t)ch.sep_cols_parent[0] * Gp, Gp, ch.R->kmin[col],
                (uint64_t)range, dense, link); c.launches++;
            GJ_CUDA_TRY(cudaGetLastError());
            dfree(c, dense);
            return cudaSuccess;
        }
    }
    k_link_search<<<grid_for(c, Gp), ST, 0, c.stream>>>(key_cols(t, ch.sep_cols_parent), Gp,
                                                        key_cols(ch, ch.sep_cols), ch.seg_first,
                                                        ch.S_dev, link); c.launches++;
    return cudaGetLastError();
}

}  // namespace

void tri_free(Ctx &c, QueryState &q);
gj_status tri_summarize(QueryState &q, uint64_t *total_out);

void query_free_summary(Ctx &c, QueryState &q) {
    tri_free(c, q);
    for (auto &t : q.r) {
        dfree(c, t.S_dev);
        dfree(c, t.L_dev);
        dfree(c, t.seg_id);
        dfree(c, t.seg_first);
        for (auto &l : t.link) dfree(c, l);
        t.link.clear();
        dfree(c, t.w);
        dfree(c, t.off);
        dfree(c, t.msg);
        dfree(c, t.down);
        dfree(c, t.mult);
        dfree(c, t.lgid);
        dfree(c, t.loff);
        dfree(c, t.lw);
        dfree(c, t.lseg_first);
    }
    q.summarized = false;
}

gj_status summarize(QueryState &q, uint64_t *total_out) {
    if (q.tri) return tri_summarize(q, total_out);
    Ctx &c = q.ctx();
    query_free_summary(c, q);
    cudaError_t e = cudaSuccess;
#define TRY(x)                                                 \
    do {                                                       \
        e = (x);                                               \
        if (e != cudaSuccess) {                                \
            note_cuda_error(e, __FILE__, __LINE__);            \
            goto fail;                                         \
        }                                                      \
    } while (0)
    {
        // segments of every non-root relation, then links parent -> child
        for (int i = 1; i < q.k; i++) TRY(build_segments(c, q.r[i]));
        for (int i = 0; i < q.k; i++) {
            QRel &t = q.r[i];
            t.link.assign(t.children.size(), nullptr);
            for (size_t ci = 0; ci < t.children.size(); ci++)
                TRY(build_link(c, t, q.r[t.children[ci]], &t.link[ci]));
        }
        // upward, leaves to root (reverse preorder)
        uint64_t *total_dev = nullptr;
        TRY(dalloc(c, &total_dev, 1));
        for (int pi = q.k - 1; pi >= 0; pi--) {
            QRel &t = q.r[q.pre[pi]];
            const int64_t G = t.F->G;
            ChildSet cs{};
            cs.n = (int)t.children.size();
            for (int ci = 0; ci < cs.n; ci++) {
                cs.link[ci] = t.link[ci];
                cs.msg[ci] = q.r[t.children[ci]].msg;
            }
            TRY(dalloc(c, &t.w, G));
            TRY(dalloc(c, &t.off, G));
            k_weights<<<grid_for(c, G), ST, 0, c.stream>>>(t.F->gstart, G, cs, t.w); c.launches++;
            TRY(cudaGetLastError());
            if (t.parent >= 0) {
                uint8_t *heads = nullptr;
                TRY(dalloc(c, &heads, G));
                k_seg_heads<<<grid_for(c, G), ST, 0, c.stream>>>(key_cols(t, t.sep_cols), G, heads); c.launches++;
                TRY(dalloc(c, &t.msg, G));      // S <= G segments
                TRY(scan_u64_sat(c, t.w, heads, t.off, G, nullptr, t.msg, t.seg_id));
                dfree(c, heads);
            } else {
                TRY(scan_u64_sat(c, t.w, nullptr, t.off, G, total_dev, nullptr, nullptr));
            }
        }
        // downward, root to leaves (preorder)
        for (int pi = 0; pi < q.k; pi++) {
            QRel &t = q.r[q.pre[pi]];
            const int64_t G = t.F->G;
            const uint64_t *t_down = t.parent >= 0 ? t.down : nullptr;
            TRY(dalloc(c, &t.mult, G));
            k_mult<<<grid_for(c, G), ST, 0, c.stream>>>(t.w, t_down, t.seg_id, G, t.mult); c.launches++;
            if (t.children.empty()) continue;
            ChildSet cs{};
            cs.n = (int)t.children.size();
            std::vector<unsigned long long *> los(cs.n);
            std::vector<unsigned int *> carries(cs.n);
            for (int ci = 0; ci < cs.n; ci++) {
                QRel &ch = q.r[t.children[ci]];
                const int64_t Sc = std::max<int64_t>(ch.F->G, 1);
                cs.link[ci] = t.link[ci];
                cs.msg[ci] = ch.msg;
                TRY(dalloc(c, &los[ci], Sc));
                TRY(dalloc(c, &carries[ci], Sc));
                TRY(cudaMemsetAsync(los[ci], 0, 8 * Sc, c.stream));
                TRY(cudaMemsetAsync(carries[ci], 0, 4 * Sc, c.stream));
                cs.lo[ci] = los[ci];
                cs.carry[ci] = carries[ci];
            }
            k_down_contrib<<<grid_for(c, G), ST, 0, c.stream>>>(t.F->gstart, G, t_down, t.seg_id, cs); c.launches++;
            TRY(cudaGetLastError());
            for (int ci = 0; ci < cs.n; ci++) {
                QRel &ch = q.r[t.children[ci]];
                TRY(dalloc(c, &ch.down, ch.F->G));
                k_down_finalize<<<grid_for(c, ch.F->G), ST, 0, c.stream>>>(los[ci], carries[ci],
                                                                         ch.S_dev, ch.down); c.launches++;
                dfree(c, los[ci]);
                dfree(c, carries[ci]);
            }
        }
        // live groups (w > 0), the only ones a result row can use
        for (int i = 0; i < q.k; i++) {
            QRel &t = q.r[i];
            const int64_t G = t.F->G;
            uint8_t *f = nullptr;
            uint32_t *lidx = nullptr;
            TRY(dalloc(c, &f, G));
            TRY(dalloc(c, &lidx, G));
            TRY(dalloc(c, &t.L_dev, 1));
            k_nonzero<<<grid_for(c, G), ST, 0, c.stream>>>(t.w, G, f); c.launches++;
            TRY(scan_u32(c, nullptr, f, lidx, G, t.L_dev));
            TRY(dalloc(c, &t.lgid, G));        // L <= G live groups
            TRY(dalloc(c, &t.loff, G));
            TRY(dalloc(c, &t.lw, G));
            k_live_compact<<<grid_for(c, G), ST, 0, c.stream>>>(f, lidx, t.w, t.off, G, t.lgid,
                                                                t.loff, t.lw); c.launches++;
            if (t.parent >= 0) {
                TRY(dalloc(c, &t.lseg_first, G + 1));
                k_live_segs<<<grid_for(c, G), ST, 0, c.stream>>>(t.seg_first, lidx, t.S_dev,
                                                                t.L_dev, t.lseg_first); c.launches++;
            }
            TRY(cudaGetLastError());
            dfree(c, f);
            dfree(c, lidx);
        }
        // the one synchronisation: |Q| and the device error word
        {
            uint64_t *h = c.pinned;
            h[0] = 0;
            if (q.r[0].F->G) TRY(cudaMemcpyAsync(h, total_dev, 8, cudaMemcpyDeviceToHost, c.stream));
            TRY(cudaMemcpyAsync(h + 1, c.err, 4, cudaMemcpyDeviceToHost, c.stream));
            TRY(cudaStreamSynchronize(c.stream));
            q.total = h[0];
            uint32_t err = (uint32_t)(h[1] & 0xffffffffu);
            dfree(c, total_dev);
            if (err) {
                cudaMemsetAsync(c.err, 0, 4, c.stream);
                return (err & ERRF_TIMEOUT) ? GJ_ERR_TIMEOUT : GJ_ERR_CUDA;
            }
        }
        q.overflow = (q.total == SAT);
    }
#undef TRY
    q.summarized = true;
    *total_out = q.total;
    return q.overflow ? GJ_ERR_OVERFLOW : GJ_OK;
fail:
    return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
}

}  // namespace gj
