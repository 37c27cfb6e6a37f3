// gj_cycle.cu -- the cyclic 3-way join R(A,B) |><| S(B,C) |><| T(C,A).
//
// A cycle has no join tree.  The paper turns the query graph into a
// junction tree whose maxcliques may hold potentials from several tables
// and joins those into one potential per maxclique (Section 3.2.1,
// Algorithm 1; inference on graphs, Section 3.4).  For three relations
// pairwise sharing one attribute there is one maxclique {A, B, C}, and its
// joint potential is the summary: every triple of groups (g_R, g_S, g_T)
// with g_R = (a, b), g_S = (b, c), g_T = (c, a), with frequency
// cnt_R * cnt_S * cnt_T (the paper's example: entries (a1,b1,5),
// (b1,c1,10), (c1,a1,20) give (a1,b1,c1,1000)).  These triples are exactly
// the blocks the desummarise emit kernel expands (rows of a block ordered by
// r_R, r_S, r_T, the last fastest), so the cyclic query reuses it unchanged.
//
// The cluster potential is built from the sorted factors, in result order,
// by sorted-list intersection (one warp per R group (a, b), R's factor
// order):
//   * S's factor is ordered by (b, c) and T's by (a, c), so the S groups with
//     key b and the T groups with key a are two segments sorted by c;
//   * the warp walks the shorter segment in c order and binary-searches the
//     longer one: every c found in both closes the cycle;
//   * a first pass counts each R group's triples, an exclusive scan places
//     them, and a second pass writes every block's three groups and its row
//     count (saturating product) in c order (ballots keep the lanes' order);
//     a saturating scan gives the blocks' first rows and |Q|.
// R groups come in R's order and each one's triples in c order, so blocks
// are ordered by (V_0, V_1, c) with V the root's columns then C.
//
// When C's value range is small next to the segments, the same triples come
// from bitmaps instead: one row per b holding S's c values, one row per a
// holding T's; an R group's triples are the set bits of the AND of its two
// rows, in c order, and a bit's rank among its row's set bits is the group's
// offset inside the segment.  Each lane takes one 32-bit word of the AND per
// step; output slots are handed to lanes in order (a search over the
// lanes' prefix counts, then a select of the bit), so the writes stay
// contiguous.
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
    const int32_t *c2, *a2;         // T's groups, ordered by (a, c)
    const uint32_t *gs2;
    int64_t G2;
};

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

// the segments of R group i: S groups with key b, T groups with key a
__device__ __forceinline__ void tri_segments(const TriSpec &s, int64_t i, uint32_t &sl, uint32_t &sh,
                                             uint32_t &tl, uint32_t &th) {
    const int32_t a = s.a0[i], b = s.b0[i];
    sl = lower_i32(s.b1, 0, (uint32_t)s.G1, b);
    sh = upper_i32(s.b1, sl, (uint32_t)s.G1, b);
    tl = lower_i32(s.a2, 0, (uint32_t)s.G2, a);
    th = upper_i32(s.a2, tl, (uint32_t)s.G2, a);
}

// One lane's element k of R group i's shorter segment and its partner in
// the other one: true if both hold the same c.  *j gets the S group, *t the
// T group.
__device__ __forceinline__ bool tri_match(const TriSpec &s, bool walk_s, uint32_t k, uint32_t sl,
                                          uint32_t sh, uint32_t tl, uint32_t th, uint32_t *j,
                                          uint32_t *t) {
    if (walk_s) {
        const uint32_t jj = sl + k;
        const int32_t c = s.c1[jj];
        const uint32_t tt = lower_i32(s.c2, tl, th, c);
        *j = jj;
        *t = tt;
        return tt < th && s.c2[tt] == c;
    }
    const uint32_t tt = tl + k;
    const int32_t c = s.c2[tt];
    const uint32_t jj = lower_i32(s.c1, sl, sh, c);
    *j = jj;
    *t = tt;
    return jj < sh && s.c1[jj] == c;
}

constexpr int TRI_WARPS = CT / 32;

// Bitmap form of S and T (rows of `words` 32-bit words; bit c - cmin of
// row x set iff the relation has the group (x + row min, c)); seg_* hold
// the first group of each row that has one.
struct TriBits {
    const uint32_t *bs, *bt;
    const uint32_t *seg_s, *seg_t;
    int32_t bmin, bmax;   // S's B values: rows of bs
    int32_t amin, amax;   // T's A values: rows of bt
    uint32_t words;
};

// rows of one relation's bitmap from its groups (ordered by row key, then c)
__global__ void k_tri_bitmap(const int32_t *__restrict__ row_key, const int32_t *__restrict__ c_key,
                             int64_t G, int32_t rmin, int32_t cmin, uint32_t words, uint32_t *bm,
                             uint32_t *seg) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rk = row_key[g];
        const uint32_t r = (uint32_t)((int64_t)rk - rmin);
        const uint32_t c = (uint32_t)((int64_t)c_key[g] - cmin);
        atomicOr(&bm[(size_t)r * words + (c >> 5)], 1u << (c & 31));
        if (g == 0 || row_key[g - 1] != rk) seg[r] = (uint32_t)g;
    }
}

// position of the r-th (from 0) set bit of m, which has more than r
__device__ __forceinline__ uint32_t select_bit(uint32_t m, uint32_t r) {
    uint32_t pos = 0;
#pragma unroll
    for (int w = 16; w; w >>= 1) {
        const uint32_t lo = __popc(m & ((1u << w) - 1u));
        if (r >= lo) {
            r -= lo;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// exclusive warp prefix sum of x; *total gets the warp's sum
__device__ __forceinline__ uint32_t warp_excl(uint32_t x, int lane, uint32_t *total) {
    uint32_t v = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += y;
    }
    *total = __shfl_sync(0xffffffffu, v, 31);
    return v - x;
}

// one warp per R group: pass WRITE=false counts its triples (cnt, total),
// WRITE=true writes its blocks from base[i] on, in c order
template <bool WRITE>
__global__ void k_tri_bits(TriSpec s, TriBits t, uint32_t *cnt, unsigned long long *total,
                           const uint32_t *__restrict__ base, uint32_t *g0, uint32_t *g1, uint32_t *g2,
                           uint64_t *W) {
    const int lane = threadIdx.x & 31;
    unsigned long long mine = 0;
    for (int64_t i = (int64_t)blockIdx.x * TRI_WARPS + (threadIdx.x >> 5); i < s.G0;
         i += (int64_t)gridDim.x * TRI_WARPS) {
        const int32_t a = s.a0[i], b = s.b0[i];
        uint32_t hits = 0;
        if (b >= t.bmin && b <= t.bmax && a >= t.amin && a <= t.amax) {
            const uint32_t rb = (uint32_t)((int64_t)b - t.bmin), ra = (uint32_t)((int64_t)a - t.amin);
            const uint32_t *rs = t.bs + (size_t)rb * t.words, *rt = t.bt + (size_t)ra * t.words;
            if (!WRITE) {
                for (uint32_t w = lane; w < t.words; w += 32) hits += __popc(rs[w] & rt[w]);
            } else {
                const uint32_t js = t.seg_s[rb], jt = t.seg_t[ra];
                const uint64_t c0 = s.gs0[i + 1] - s.gs0[i];
                uint32_t at = base[i], sr = 0, tr = 0;   // slots, S bits, T bits so far
                for (uint32_t w0 = 0; w0 < t.words; w0 += 32) {
                    const uint32_t w = w0 + lane;
                    const uint32_t sw = w < t.words ? rs[w] : 0u, tw = w < t.words ? rt[w] : 0u;
                    const uint32_t x = sw & tw;
                    uint32_t ns, nt, nx;
                    const uint32_t es = warp_excl(__popc(sw), lane, &ns);
                    const uint32_t et = warp_excl(__popc(tw), lane, &nt);
                    const uint32_t ex = warp_excl(__popc(x), lane, &nx);
                    for (uint32_t o0 = 0; o0 < nx; o0 += 32) {
                        const uint32_t o = o0 + lane;
                        // the lane whose word holds slot o: the last one with ex <= o
                        uint32_t L = 0;
#pragma unroll
                        for (int st = 16; st; st >>= 1) {
                            const uint32_t e = __shfl_sync(0xffffffffu, ex, L + st);
                            if (e <= o) L += st;
                        }
                        const uint32_t xL = __shfl_sync(0xffffffffu, x, L);
                        const uint32_t exL = __shfl_sync(0xffffffffu, ex, L);
                        const uint32_t swL = __shfl_sync(0xffffffffu, sw, L);
                        const uint32_t esL = __shfl_sync(0xffffffffu, es, L);
                        const uint32_t twL = __shfl_sync(0xffffffffu, tw, L);
                        const uint32_t etL = __shfl_sync(0xffffffffu, et, L);
                        if (o < nx) {
                            const uint32_t bit = select_bit(xL, o - exL);
                            const uint32_t below = (1u << bit) - 1u;
                            const uint32_t j = js + sr + esL + __popc(swL & below);
                            const uint32_t k = jt + tr + etL + __popc(twL & below);
                            const uint32_t slot = at + o;
                            g0[slot] = (uint32_t)i;
                            g1[slot] = j;
                            g2[slot] = k;
                            const uint64_t c1 = s.gs1[j + 1] - s.gs1[j], c2 = s.gs2[k + 1] - s.gs2[k];
                            W[slot] = sat_mul(sat_mul(c0, c1), c2);
                        }
                    }
                    at += nx;
                    sr += ns;
                    tr += nt;
                }
            }
        }
        if (!WRITE) {
            hits = __reduce_add_sync(0xffffffffu, hits);
            if (lane == 0) {
                cnt[i] = hits;
                mine += hits;
            }
        }
    }
    if (!WRITE && lane == 0 && mine) atomicAdd(total, mine);
}

// pass 1: triples per R group (a warp per group) and their exact total
__global__ void k_tri_count(TriSpec s, uint32_t *cnt, unsigned long long *total) {
    const int lane = threadIdx.x & 31;
    unsigned long long mine = 0;
    for (int64_t i = (int64_t)blockIdx.x * TRI_WARPS + (threadIdx.x >> 5); i < s.G0;
         i += (int64_t)gridDim.x * TRI_WARPS) {
        uint32_t sl, sh, tl, th;
        tri_segments(s, i, sl, sh, tl, th);
        const bool walk_s = sh - sl <= th - tl;
        const uint32_t len = (sl == sh || tl == th) ? 0 : (walk_s ? sh - sl : th - tl);
        uint32_t hits = 0;
        for (uint32_t k0 = 0; k0 < len; k0 += 32) {
            uint32_t j, t;
            const bool hit = k0 + lane < len && tri_match(s, walk_s, k0 + lane, sl, sh, tl, th, &j, &t);
            hits += __popc(__ballot_sync(0xffffffffu, hit));
        }
        if (lane == 0) { cnt[i] = hits; mine += hits; }
    }
    if (lane == 0 && mine) atomicAdd(total, mine);
}

// pass 2: R group i's blocks at base[i] onwards, in c order
__global__ void k_tri_blocks(TriSpec s, const uint32_t *__restrict__ base, uint32_t *g0, uint32_t *g1,
                             uint32_t *g2, uint64_t *W) {
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    for (int64_t i = (int64_t)blockIdx.x * TRI_WARPS + (threadIdx.x >> 5); i < s.G0;
         i += (int64_t)gridDim.x * TRI_WARPS) {
        uint32_t sl, sh, tl, th;
        tri_segments(s, i, sl, sh, tl, th);
        const bool walk_s = sh - sl <= th - tl;
        const uint32_t len = (sl == sh || tl == th) ? 0 : (walk_s ? sh - sl : th - tl);
        uint32_t at = base[i];
        const uint64_t c0 = s.gs0[i + 1] - s.gs0[i];
        for (uint32_t k0 = 0; k0 < len; k0 += 32) {
            uint32_t j = 0, t = 0;
            const bool hit = k0 + lane < len && tri_match(s, walk_s, k0 + lane, sl, sh, tl, th, &j, &t);
            const uint32_t m = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const uint32_t b = at + __popc(m & below);
                g0[b] = (uint32_t)i;
                g1[b] = j;
                g2[b] = t;
                const uint64_t c1 = s.gs1[j + 1] - s.gs1[j], c2 = s.gs2[t + 1] - s.gs2[t];
                W[b] = sat_mul(sat_mul(c0, c1), c2);
            }
            at += __popc(m);
        }
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

// Bitmap plan for the query's factors, or false when the lists are the
// better (or the only affordable) form.  mode: 0 chooses, 1 lists, 2 bitmaps
// when they fit.
constexpr int64_t TRI_BITS_BYTES = 512ll << 20;

bool tri_bits_plan(QueryState &q, const TriSpec &s, int mode, TriBits &t, int64_t &rows_s,
                   int64_t &rows_t) {
    if (mode == 1) return false;
    const Relation &RS = *q.r[1].R, &RT = *q.r[2].R;
    const int sb = q.tri_col[1][0], sc = q.tri_col[1][1];
    const int tc = q.tri_col[2][0], ta = q.tri_col[2][1];
    rows_s = (int64_t)RS.kmax[sb] - RS.kmin[sb] + 1;
    rows_t = (int64_t)RT.kmax[ta] - RT.kmin[ta] + 1;
    const int64_t cmin = std::min(RS.kmin[sc], RT.kmin[tc]), cmax = std::max(RS.kmax[sc], RT.kmax[tc]);
    const int64_t words = (cmax - cmin + 1 + 31) / 32;
    if ((rows_s + rows_t) * (words + 1) * 4 > TRI_BITS_BYTES) return false;
    if (mode == 0) {
        // a warp step of the bitmaps covers 1024 values of c; one of the lists
        // covers 32 groups of the shorter segment, each with a binary search
        const double seg_s = (double)s.G1 / (double)rows_s, seg_t = (double)s.G2 / (double)rows_t;
        if ((double)((words + 31) / 32) > 1.0 + std::min(seg_s, seg_t) / 8.0) return false;
    }
    t.bmin = RS.kmin[sb];
    t.bmax = RS.kmax[sb];
    t.amin = RT.kmin[ta];
    t.amax = RT.kmax[ta];
    t.words = (uint32_t)words;
    (void)cmax;
    return true;
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
    uint32_t *hits = nullptr, *base = nullptr, *cnt = nullptr;
    uint32_t *bm = nullptr, *seg = nullptr;
    uint64_t *W = nullptr, *total_dev = nullptr;
    TriBits tb{};
    int64_t rows_s = 0, rows_t = 0;
    bool bits = false;
    unsigned long long *tsum = nullptr;
    unsigned long long nb = 0;
    uint64_t total = 0;
    gj_status st = GJ_OK;
    cudaError_t e = cudaSuccess;
    const int64_t warps_grid = std::max<int64_t>(
        1, std::min<int64_t>(ceil_div(s.G0, TRI_WARPS), (int64_t)c.num_sms * 16));
    auto groups_grid = [&](int64_t n) {
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, CT), (int64_t)c.num_sms * 16));
    };
#define TRY(x)                                                 \
    do {                                                       \
        e = (x);                                               \
        if (e != cudaSuccess) {                                \
            note_cuda_error(e, __FILE__, __LINE__);            \
            goto fail;                                         \
        }                                                      \
    } while (0)
    TRY(dalloc(c, &cnt, 1));
    TRY(dalloc(c, &total_dev, 1));
    TRY(dalloc(c, &tsum, 1));
    TRY(cudaMemsetAsync(tsum, 0, sizeof(unsigned long long), c.stream));
    if (s.G0 > 0 && s.G1 > 0 && s.G2 > 0) {
        // triples per R group, placed by a scan
        TRY(dalloc(c, &hits, s.G0));
        TRY(dalloc(c, &base, s.G0));
        bits = tri_bits_plan(q, s, c.tri_mode, tb, rows_s, rows_t);
        if (bits) {
            const size_t nbits = (size_t)(rows_s + rows_t) * tb.words;
            TRY(dalloc(c, &bm, nbits));
            TRY(dalloc(c, &seg, (size_t)(rows_s + rows_t)));
            TRY(cudaMemsetAsync(bm, 0, nbits * 4, c.stream));
            TRY(cudaMemsetAsync(seg, 0, (size_t)(rows_s + rows_t) * 4, c.stream));
            const Relation &RS = *q.r[1].R, &RT = *q.r[2].R;
            const int32_t cmin = std::min(RS.kmin[q.tri_col[1][1]], RT.kmin[q.tri_col[2][0]]);
            tb.bs = bm;
            tb.bt = bm + (size_t)rows_s * tb.words;
            tb.seg_s = seg;
            tb.seg_t = seg + rows_s;
            k_tri_bitmap<<<groups_grid(s.G1), CT, 0, c.stream>>>(s.b1, s.c1, s.G1, tb.bmin, cmin, tb.words,
                                                                  bm, seg); c.launches++;
            k_tri_bitmap<<<groups_grid(s.G2), CT, 0, c.stream>>>(s.a2, s.c2, s.G2, tb.amin, cmin, tb.words,
                                                                  bm + (size_t)rows_s * tb.words,
                                                                  seg + rows_s); c.launches++;
            k_tri_bits<false><<<(unsigned)warps_grid, CT, 0, c.stream>>>(s, tb, hits, tsum, nullptr, nullptr,
                                                                        nullptr, nullptr, nullptr); c.launches++;
        } else {
            k_tri_count<<<(unsigned)warps_grid, CT, 0, c.stream>>>(s, hits, tsum); c.launches++;
        }
        TRY(cudaGetLastError());
        TRY(readback(c, tsum, &nb, 8));
        // blocks are numbered in 32 bits
        if (nb > 0x7fffffffull) { st = GJ_ERR_CAPACITY; goto done; }
        if (nb > 0) {
            TRY(scan_u32(c, hits, nullptr, base, s.G0, cnt));
            for (auto &g : q.blk_grp) TRY(dalloc(c, &g, nb));
            TRY(dalloc(c, &W, nb));
            TRY(dalloc(c, &q.blk_A, nb));
            if (bits)
                k_tri_bits<true><<<(unsigned)warps_grid, CT, 0, c.stream>>>(
                    s, tb, nullptr, nullptr, base, q.blk_grp[0], q.blk_grp[1], q.blk_grp[2], W);
            else
                k_tri_blocks<<<(unsigned)warps_grid, CT, 0, c.stream>>>(s, base, q.blk_grp[0], q.blk_grp[1],
                                                                        q.blk_grp[2], W);
            c.launches++;
            TRY(cudaGetLastError());
            TRY(scan_u64_sat(c, W, nullptr, q.blk_A, (int64_t)nb, total_dev, nullptr, nullptr));
            TRY(readback(c, total_dev, &total, 8));
        }
    }
    st = check_device_error(c);
    if (st != GJ_OK) goto done;
    q.nblocks = nb;
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
    dfree(c, hits);
    dfree(c, base);
    dfree(c, bm);
    dfree(c, seg);
    dfree(c, cnt);
    dfree(c, W);
    dfree(c, total_dev);
    dfree(c, tsum);
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
