// gj_batch.cu -- many independent join queries summarised together.
//
// Each query's summary is the upward pass of Algorithm 2 (Section 3.3):
// per relation the frequency table (Section 3.2), per group
// w = cnt (x) prod_children msg, per separator value msg = (+) w, and at the
// root |Q| = (+) w.  Run one query at a time, a query of 3-6 small tables
// costs tens of launches and several host synchronisations, which dominate.
// Here the relations of ALL queries are processed by one fixed sequence of
// kernels with no host synchronisation, so the sequence can be captured in
// a CUDA graph and replayed as one launch:
//
//   plan    (host, once)   join tree of every query; relations renumbered
//                          deepest level first, so every tree level is a
//                          contiguous slice of relations, of rows and (after
//                          sorting) of groups; per-relation min/max (the only
//                          synchronisation) fixes the key packing.
//   pack                   key = (relation, separator value, other value)
//   sort                   one keys-only LSD radix sort over all rows
//   heads + scans          group ids and segment ids (segments = equal
//                          relation and separator value)
//   groups                 group starts, group -> segment, and a dense
//                          value -> segment table per relation
//   levels, deepest first  persistent kernels over the level's group slice
//                          (bounds read from device memory): w of every
//                          group, summed into its segment's message (or its
//                          query's total at the root) by saturating atomics,
//                          aggregated across each warp's runs of equal target
//   totals                 |Q| and status per query
//
// The batched kernels take relations of one or two key columns whose
// non-root relations share exactly one attribute with their parent.  Other
// queries of a batch (three or more key columns, separators of several
// attributes) are summarised through the single-query path by gj_batch_run,
// after the batched kernels, and report their totals and statuses in the
// same arrays.
#include <string.h>

#include <algorithm>

#include "gj_state.cuh"

namespace gj {

cudaError_t radix_sort_keys_prepare();
cudaError_t radix_sort_keys_u64_in(Ctx &c, uint64_t *keys, int64_t n, int bits, uint64_t *k2,
                                   uint32_t *hist, unsigned long long *status,
                                   int64_t status_tiles);
cudaError_t scan_u32_in(Ctx &c, const uint32_t *in, const uint8_t *flags, uint32_t *out,
                        int64_t n, uint32_t *total_dev, void *state_mem, size_t state_bytes);
size_t scan_u32_state_bytes(int64_t n);
gj_status check_device_error(Ctx &c);

namespace {

constexpr int BT = 256;
constexpr int BMAXCH = MAX_REL;           // children per relation in a batch
constexpr int64_t PACK_TILE = 4096;

// per batch relation, device side
struct BRel {
    const int32_t *col_a;    // separator column (root: first declared column)
    const int32_t *col_b;    // other column or NULL
    int32_t min_a, min_b;
    int32_t query;
    int32_t is_root;
    int32_t nchild;
    int32_t child[BMAXCH];
    int32_t child_pcol[BMAXCH];   // 0: child's separator is this relation's a, 1: its b
    int64_t doff;                 // dense table offset (non-root)
    uint32_t range;               // dense table size (non-root)
};

struct BKeys {
    int bits_a, bits_b;
    uint64_t mask_a, mask_b;
};

// relation field of a packed key (empty when the value fields fill 64 bits,
// which planning allows only for a single relation)
__device__ __forceinline__ uint32_t key_rel(const BKeys &k, uint64_t key) {
    int s = k.bits_a + k.bits_b;
    return s >= 64 ? 0u : (uint32_t)(key >> s);
}

__global__ void __launch_bounds__(BT) k_bminmax(const BRel *rels, const int64_t *roff, int32_t *mm) {
    const int b = blockIdx.x;
    const BRel R = rels[b];
    int32_t a_lo = INT32_MAX, a_hi = INT32_MIN, b_lo = INT32_MAX, b_hi = INT32_MIN;
    for (int64_t i = roff[b] + threadIdx.x; i < roff[b + 1]; i += BT) {
        int32_t x = R.col_a[i - roff[b]];
        a_lo = min(a_lo, x);
        a_hi = max(a_hi, x);
        if (R.col_b) {
            int32_t y = R.col_b[i - roff[b]];
            b_lo = min(b_lo, y);
            b_hi = max(b_hi, y);
        }
    }
    for (int d = 16; d; d >>= 1) {
        a_lo = min(a_lo, __shfl_xor_sync(0xffffffffu, a_lo, d));
        a_hi = max(a_hi, __shfl_xor_sync(0xffffffffu, a_hi, d));
        b_lo = min(b_lo, __shfl_xor_sync(0xffffffffu, b_lo, d));
        b_hi = max(b_hi, __shfl_xor_sync(0xffffffffu, b_hi, d));
    }
    __shared__ int32_t s[4][BT / 32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s[0][w] = a_lo; s[1][w] = a_hi; s[2][w] = b_lo; s[3][w] = b_hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < BT / 32; i++) {
            a_lo = min(a_lo, s[0][i]); a_hi = max(a_hi, s[1][i]);
            b_lo = min(b_lo, s[2][i]); b_hi = max(b_hi, s[3][i]);
        }
        if (!R.col_b) { b_lo = 0; b_hi = 0; }
        if (roff[b] == roff[b + 1]) { a_lo = a_hi = b_lo = b_hi = 0; }
        mm[4 * b] = a_lo; mm[4 * b + 1] = a_hi; mm[4 * b + 2] = b_lo; mm[4 * b + 3] = b_hi;
    }
}

__global__ void k_bpack(const BRel *__restrict__ rels, const int64_t *__restrict__ roff,
                        const int32_t *__restrict__ tile_rel, int64_t N, BKeys bk,
                        uint64_t *__restrict__ keys) {
    for (int64_t i = (int64_t)blockIdx.x * BT + threadIdx.x; i < N; i += (int64_t)gridDim.x * BT) {
        int32_t b = tile_rel[i / PACK_TILE];
        while (roff[b + 1] <= i) b++;
        const BRel &R = rels[b];
        int64_t r = i - roff[b];
        uint64_t fa = (uint32_t)R.col_a[r] - (uint32_t)R.min_a;
        uint64_t fb = R.col_b ? (uint64_t)((uint32_t)R.col_b[r] - (uint32_t)R.min_b) : 0ull;
        const int rs = bk.bits_a + bk.bits_b;
        keys[i] = (rs >= 64 ? 0ull : ((uint64_t)b << rs)) | (bk.bits_b >= 64 ? 0ull : (fa << bk.bits_b)) | fb;
    }
}

__global__ void k_bheads(const uint64_t *__restrict__ keys, int64_t N, BKeys bk,
                         uint8_t *__restrict__ ghead, uint8_t *__restrict__ shead) {
    for (int64_t i = (int64_t)blockIdx.x * BT + threadIdx.x; i < N; i += (int64_t)gridDim.x * BT) {
        uint64_t k = keys[i];
        uint8_t g = 1, s = 1;
        if (i > 0) {
            uint64_t p = keys[i - 1];
            g = k != p;
            s = (k >> bk.bits_b) != (p >> bk.bits_b);
        }
        ghead[i] = g;
        shead[i] = s;
    }
}

__global__ void k_bgroups(const uint64_t *__restrict__ keys, const uint8_t *__restrict__ ghead,
                          const uint8_t *__restrict__ shead, const uint32_t *__restrict__ gid,
                          const uint32_t *__restrict__ sid, int64_t N, BKeys bk,
                          const BRel *__restrict__ rels, uint32_t *__restrict__ gstart,
                          uint32_t *__restrict__ gsid, uint32_t *__restrict__ dense,
                          uint32_t *err) {
    for (int64_t i = (int64_t)blockIdx.x * BT + threadIdx.x; i < N; i += (int64_t)gridDim.x * BT) {
        const uint32_t s = sid[i] + shead[i] - 1u;
        if (ghead[i]) {
            uint32_t g = gid[i];
            gstart[g] = (uint32_t)i;
            gsid[g] = s;
        }
        if (shead[i]) {
            uint64_t k = keys[i];
            uint32_t b = key_rel(bk, k);
            const BRel &R = rels[b];
            if (!R.is_root) {
                uint64_t fa = (k >> bk.bits_b) & bk.mask_a;
                if (fa < R.range) dense[R.doff + fa] = s;
                else raise_err(err, ERRF_BOUNDS);
            }
        }
        if (i == N - 1) gstart[gid[i] + ghead[i]] = (uint32_t)N;
    }
}

// first group / segment of every relation (relation R = the end)
__global__ void k_brel_bounds(const int64_t *roff, int R, int64_t N, const uint32_t *gid,
                              const uint32_t *sid, const uint32_t *gcount, const uint32_t *scount,
                              uint32_t *rel_gbeg, uint32_t *rel_sbeg) {
    for (int b = blockIdx.x * BT + threadIdx.x; b <= R; b += gridDim.x * BT) {
        int64_t r = roff[b];
        rel_gbeg[b] = r < N ? gid[r] : *gcount;
        rel_sbeg[b] = r < N ? sid[r] : *scount;
    }
}

__device__ __forceinline__ void sat_atomic_add(unsigned long long *lo, unsigned int *carry,
                                               uint64_t x) {
    if (x == 0) return;
    if (x == SAT) { atomicOr(carry, 1u); return; }
    unsigned long long old = atomicAdd(lo, (unsigned long long)x);
    if (old + x < old) atomicOr(carry, 1u);
}

// w of every group of one level; summed per target (segment, or query at
// the root).  Targets do not decrease across a warp's consecutive groups,
// so each run of equal targets is reduced with shuffles and added once.
__global__ void __launch_bounds__(BT)
k_bweights(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ gstart,
           const uint32_t *__restrict__ gsid, const uint32_t *__restrict__ rel_gbeg, int lr_beg,
           int lr_end, BKeys bk, const BRel *__restrict__ rels, const uint32_t *__restrict__ dense,
           const uint64_t *__restrict__ msg, unsigned long long *msg_lo, unsigned int *msg_carry,
           unsigned long long *tot_lo, unsigned int *tot_carry) {
    const int64_t gbeg = rel_gbeg[lr_beg], gend = rel_gbeg[lr_end];
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * BT;
    for (int64_t base = gbeg + (int64_t)blockIdx.x * BT; base < gend; base += stride) {
        const int64_t g = base + threadIdx.x;
        uint64_t w = 0;
        uint64_t target = ~0ull;     // (is_root << 63) | index, or none
        if (g < gend) {
            const uint32_t i0 = gstart[g];
            const uint64_t key = keys[i0];
            const uint32_t b = key_rel(bk, key);
            const BRel &R = rels[b];
            w = (uint64_t)(gstart[g + 1] - i0);
            const uint64_t fa = (key >> bk.bits_b) & bk.mask_a, fb = key & bk.mask_b;
            for (int ci = 0; ci < R.nchild; ci++) {
                const int c = R.child[ci];
                const BRel &C = rels[c];
                int32_t v = R.child_pcol[ci] == 0 ? (int32_t)((uint32_t)fa + (uint32_t)R.min_a)
                                                  : (int32_t)((uint32_t)fb + (uint32_t)R.min_b);
                uint32_t idx = (uint32_t)v - (uint32_t)C.min_a;
                uint32_t s = idx < C.range ? dense[C.doff + idx] : NONE;
                w = sat_mul(w, s == NONE ? 0ull : msg[s]);
            }
            target = R.is_root ? ((1ull << 63) | (uint64_t)R.query) : (uint64_t)gsid[g];
        }
        // segmented inclusive scan of w over runs of equal target
        uint64_t run = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t ov = __shfl_up_sync(0xffffffffu, run, d);
            uint64_t ot = __shfl_up_sync(0xffffffffu, target, d);
            if (lane >= d && ot == target) run = sat_add(ov, run);
        }
        uint64_t next_t = __shfl_down_sync(0xffffffffu, target, 1);
        bool last = (lane == 31) || next_t != target;
        if (last && target != ~0ull && run != 0) {
            if (target >> 63) {
                uint64_t q = target & ~(1ull << 63);
                sat_atomic_add(tot_lo + q, tot_carry + q, run);
            } else {
                sat_atomic_add(msg_lo + target, msg_carry + target, run);
            }
        }
    }
}

__global__ void k_bfinalize(const uint32_t *__restrict__ rel_sbeg, int lr_beg, int lr_end,
                            unsigned long long *msg_lo, const unsigned int *msg_carry) {
    const int64_t sbeg = rel_sbeg[lr_beg], send = rel_sbeg[lr_end];
    for (int64_t s = sbeg + (int64_t)blockIdx.x * BT + threadIdx.x; s < send;
         s += (int64_t)gridDim.x * BT) {
        if (msg_carry[s] || msg_lo[s] == SAT) msg_lo[s] = SAT;
    }
}

__global__ void k_btotals(const unsigned long long *tot_lo, const unsigned int *tot_carry, int Q,
                          uint64_t *totals, int32_t *status) {
    for (int q = blockIdx.x * BT + threadIdx.x; q < Q; q += gridDim.x * BT) {
        uint64_t t = (tot_carry[q] || tot_lo[q] == SAT) ? SAT : (uint64_t)tot_lo[q];
        totals[q] = t;
        if (status) status[q] = t == SAT ? (int32_t)GJ_ERR_OVERFLOW : (int32_t)GJ_OK;
    }
}

inline int bits_of(uint64_t range) { return range == 0 ? 0 : 64 - __builtin_clzll(range); }

}  // namespace

struct BatchState {
    CtxState *cs = nullptr;
    int Q = 0, R = 0, levels = 0;
    int64_t N = 0, S_cap = 0, dense_size = 0;
    BKeys bk{};
    int key_bits = 0;
    std::vector<int> lr_beg, lr_end;         // relation range of level d (0 = root level)
    int grid_mult = 4;
    // device tables
    BRel *rels = nullptr;
    int64_t *roff = nullptr;
    int32_t *tile_rel = nullptr;
    // workspace
    uint64_t *keys = nullptr, *k2 = nullptr;
    uint8_t *ghead = nullptr, *shead = nullptr;
    uint32_t *gid = nullptr, *sid = nullptr, *counts = nullptr;
    void *scan_state[2] = {nullptr, nullptr};
    size_t scan_bytes = 0;
    uint32_t *hist = nullptr;
    unsigned long long *status = nullptr;
    int64_t status_tiles = 0;
    uint32_t *gstart = nullptr, *gsid = nullptr, *dense = nullptr;
    uint32_t *rel_gbeg = nullptr, *rel_sbeg = nullptr;
    unsigned long long *msg_lo = nullptr, *tot_lo = nullptr;
    unsigned int *msg_carry = nullptr, *tot_carry = nullptr;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t *g_totals = nullptr;
    int32_t *g_status = nullptr;
    int g_mult = 0;
    uint64_t g_launches = 0;   // kernels inside the captured graph
    // graphs are captured on this private stream (the context's stream may be
    // the legacy default stream, which cannot be captured) and launched on
    // the context's stream
    cudaStream_t capture_stream = nullptr;
    // queries outside the batched kernels' shapes: (query index, its query)
    std::vector<std::pair<int, gj_query *>> fallback;
    std::vector<uint64_t> fb_total;
    std::vector<int32_t> fb_status;
};

namespace {

void batch_free(BatchState &b) {
    for (auto &f : b.fallback) gj_query_destroy(f.second);
    b.fallback.clear();
    Ctx &c = b.cs->c;
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.graph) cudaGraphDestroy(b.graph);
    if (b.capture_stream) cudaStreamDestroy(b.capture_stream);
    b.capture_stream = nullptr;
    b.exec = nullptr;
    b.graph = nullptr;
    void *ptrs[] = {b.rels, b.roff, b.tile_rel, b.keys, b.k2, b.ghead, b.shead, b.gid, b.sid,
                    b.counts, b.scan_state[0], b.scan_state[1], b.hist, b.status, b.gstart,
                    b.gsid, b.dense, b.rel_gbeg, b.rel_sbeg, b.msg_lo, b.tot_lo, b.msg_carry,
                    b.tot_carry};
    for (void *p : ptrs) if (p) cudaFreeAsync(p, c.stream);
    cudaStreamSynchronize(c.stream);
}

// The whole summary of the batch: enqueued only, no synchronisation.
cudaError_t batch_enqueue(BatchState &b, Ctx &c, uint64_t *totals, int32_t *status_out) {
    const int64_t N = b.N;
    const int grid = std::max(1, c.num_sms * b.grid_mult);
    GJ_CUDA_TRY(cudaMemsetAsync(b.dense, 0xFF, sizeof(uint32_t) * std::max<int64_t>(b.dense_size, 1), c.stream));
    GJ_CUDA_TRY(cudaMemsetAsync(b.msg_lo, 0, sizeof(unsigned long long) * b.S_cap, c.stream));
    GJ_CUDA_TRY(cudaMemsetAsync(b.msg_carry, 0, sizeof(unsigned int) * b.S_cap, c.stream));
    GJ_CUDA_TRY(cudaMemsetAsync(b.tot_lo, 0, sizeof(unsigned long long) * b.Q, c.stream));
    GJ_CUDA_TRY(cudaMemsetAsync(b.tot_carry, 0, sizeof(unsigned int) * b.Q, c.stream));
    if (N > 0) {
        k_bpack<<<grid, BT, 0, c.stream>>>(b.rels, b.roff, b.tile_rel, N, b.bk, b.keys); c.launches++;
        GJ_CUDA_TRY(radix_sort_keys_u64_in(c, b.keys, N, b.key_bits, b.k2, b.hist, b.status,
                                           b.status_tiles));
        k_bheads<<<grid, BT, 0, c.stream>>>(b.keys, N, b.bk, b.ghead, b.shead); c.launches++;
        GJ_CUDA_TRY(scan_u32_in(c, nullptr, b.ghead, b.gid, N, b.counts, b.scan_state[0], b.scan_bytes));
        GJ_CUDA_TRY(scan_u32_in(c, nullptr, b.shead, b.sid, N, b.counts + 1, b.scan_state[1], b.scan_bytes));
        k_bgroups<<<grid, BT, 0, c.stream>>>(b.keys, b.ghead, b.shead, b.gid, b.sid, N, b.bk,
                                             b.rels, b.gstart, b.gsid, b.dense, c.err); c.launches++;
    } else {
        GJ_CUDA_TRY(cudaMemsetAsync(b.counts, 0, 2 * sizeof(uint32_t), c.stream));
    }
    k_brel_bounds<<<(b.R + BT) / BT, BT, 0, c.stream>>>(b.roff, b.R, N, b.gid, b.sid, b.counts,
                                                      b.counts + 1, b.rel_gbeg, b.rel_sbeg); c.launches++;
    for (int d = b.levels - 1; d >= 0; d--) {
        if (b.lr_beg[d] == b.lr_end[d]) continue;
        k_bweights<<<grid, BT, 0, c.stream>>>(b.keys, b.gstart, b.gsid, b.rel_gbeg, b.lr_beg[d],
                                              b.lr_end[d], b.bk, b.rels, b.dense,
                                              (const uint64_t *)b.msg_lo, b.msg_lo, b.msg_carry,
                                              b.tot_lo, b.tot_carry); c.launches++;
        if (d > 0) {
            k_bfinalize<<<grid, BT, 0, c.stream>>>(b.rel_sbeg, b.lr_beg[d], b.lr_end[d], b.msg_lo,
                                                   b.msg_carry); c.launches++;
        }
    }
    k_btotals<<<(b.Q + BT - 1) / BT, BT, 0, c.stream>>>(b.tot_lo, b.tot_carry, b.Q, totals,
                                                        status_out); c.launches++;
    GJ_CUDA_TRY(cudaGetLastError());
    return cudaSuccess;
}

}  // namespace
}  // namespace gj

struct gj_batch {
    gj::BatchState s;
};

using namespace gj;

extern "C" {

gj_status gj_batch_create(gj_ctx *ctx, const int32_t *rel_ids, const int32_t *query_off,
                          int32_t n_queries, gj_batch **out) {
    if (!ctx || !rel_ids || !query_off || !out || n_queries < 1) return GJ_ERR_INVALID;
    *out = nullptr;
    CtxState &cs = ctx->s;
    Ctx &c = cs.c;
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (dev_prev != c.device) cudaSetDevice(c.device);
    struct HRel {
        Relation *R;
        int q, pos, parent, depth;
        int col_a, col_b;      // sort columns in the relation
        std::vector<int> children;
        std::vector<int> child_pcol;
    };
    std::vector<HRel> hr;
    std::vector<int> qroot(n_queries);
    gj_status st = GJ_OK;
    std::vector<std::pair<int, gj_query *>> fallback;
    for (int q = 0; q < n_queries && st == GJ_OK; q++) {
        int k = query_off[q + 1] - query_off[q];
        if (k < 1 || k > MAX_REL) { st = GJ_ERR_INVALID; break; }
        int base = (int)hr.size();
        qroot[q] = base;
        std::vector<int32_t> seen;
        bool other_shape = false;   // outside the batched kernels' shapes
        for (int j = 0; j < k; j++) {
            auto it = cs.rels.find(rel_ids[query_off[q] + j]);
            if (it == cs.rels.end()) { st = GJ_ERR_INVALID; break; }
            Relation *R = it->second.get();
            if (R->nk < 1 || R->nk > 2) { other_shape = true; break; }
            HRel h{R, q, j, -1, 0, 0, R->nk == 2 ? 1 : -1, {}, {}};
            if (j > 0) {
                std::vector<int> shared_cols;
                for (int cc = 0; cc < R->nk; cc++)
                    if (std::find(seen.begin(), seen.end(), R->attr[cc]) != seen.end())
                        shared_cols.push_back(cc);
                if (shared_cols.size() != 1) { other_shape = true; break; }
                int32_t a = R->attr[shared_cols[0]];
                int parent = -1;
                for (int i = 0; i < j && parent < 0; i++) {
                    const auto &pa = hr[base + i].R->attr;
                    if (std::find(pa.begin(), pa.end(), a) != pa.end()) parent = i;
                }
                if (parent < 0) { st = GJ_ERR_NOT_ACYCLIC; break; }
                h.parent = base + parent;
                h.depth = hr[base + parent].depth + 1;
                h.col_a = shared_cols[0];
                h.col_b = R->nk == 2 ? 1 - shared_cols[0] : -1;
                HRel &P = hr[base + parent];
                if ((int)P.children.size() >= BMAXCH) { other_shape = true; break; }
                int pc = P.R->attr[P.col_a] == a ? 0 : 1;
                P.children.push_back(base + j);
                P.child_pcol.push_back(pc);
            }
            for (int32_t a : R->attr) seen.push_back(a);
            hr.push_back(h);
        }
        if (st == GJ_OK && other_shape) {
            // this query goes through the single-query path: planned (and
            // its factors built) now, summarised by gj_batch_run
            hr.resize(base);
            gj_query *fq = nullptr;
            st = gj_query_create(ctx, rel_ids + query_off[q], k, &fq);
            if (st == GJ_OK) fallback.emplace_back(q, fq);
        }
    }
    auto drop_fallback = [&]() {
        for (auto &f : fallback) gj_query_destroy(f.second);
        fallback.clear();
    };
    if (st != GJ_OK) { drop_fallback(); if (dev_prev != c.device) cudaSetDevice(dev_prev); return st; }
    // renumber: deepest level first, then query, then position
    const int Rn = (int)hr.size();
    int levels = 0;
    for (auto &h : hr) levels = std::max(levels, h.depth + 1);
    std::vector<int> order(Rn);
    for (int i = 0; i < Rn; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hr[x].depth > hr[y].depth; });
    std::vector<int> newid(Rn);
    for (int i = 0; i < Rn; i++) newid[order[i]] = i;
    std::unique_ptr<gj_batch> bb(new gj_batch());
    BatchState &b = bb->s;
    b.cs = &cs;
    b.Q = n_queries;
    b.R = Rn;
    b.levels = levels;
    b.fallback = fallback;
    fallback.clear();
    if (Rn == 0) {   // every query takes the single-query path
        if (dev_prev != c.device) cudaSetDevice(dev_prev);
        *out = bb.release();
        return GJ_OK;
    }
    b.lr_beg.assign(levels, 0);
    b.lr_end.assign(levels, 0);
    for (int d = 0; d < levels; d++) {
        int beg = Rn, end = 0;
        for (int i = 0; i < Rn; i++)
            if (hr[order[i]].depth == d) { beg = std::min(beg, i); end = std::max(end, i + 1); }
        if (beg > end) beg = end = 0;
        b.lr_beg[d] = beg;
        b.lr_end[d] = end;
    }
    std::vector<BRel> brel(Rn);
    std::vector<int64_t> roff(Rn + 1, 0);
    for (int i = 0; i < Rn; i++) {
        const HRel &h = hr[order[i]];
        BRel &x = brel[i];
        memset(&x, 0, sizeof(x));
        x.col_a = h.R->key[h.col_a];
        x.col_b = h.col_b >= 0 ? h.R->key[h.col_b] : nullptr;
        x.query = h.q;
        x.is_root = h.parent < 0;
        x.nchild = (int)h.children.size();
        for (int ci = 0; ci < x.nchild; ci++) {
            x.child[ci] = newid[h.children[ci]];
            x.child_pcol[ci] = h.child_pcol[ci];
        }
        roff[i + 1] = roff[i] + h.R->n;
    }
    b.N = roff[Rn];
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t err) {
        note_cuda_error(err, __FILE__, __LINE__);
        batch_free(b);
        if (dev_prev != c.device) cudaSetDevice(dev_prev);
        return err == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
    };
    if (b.N > 0xffffffffLL) { batch_free(b); if (dev_prev != c.device) cudaSetDevice(dev_prev); return GJ_ERR_INVALID; }
    if ((e = radix_sort_keys_prepare()) != cudaSuccess) return fail(e);
    // per-relation min/max (the one synchronisation of planning)
    if ((e = dalloc(c, &b.rels, Rn)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.roff, Rn + 1)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(b.rels, brel.data(), sizeof(BRel) * Rn, cudaMemcpyHostToDevice, c.stream))) return fail(e);
    if ((e = cudaMemcpyAsync(b.roff, roff.data(), sizeof(int64_t) * (Rn + 1), cudaMemcpyHostToDevice, c.stream))) return fail(e);
    std::vector<int32_t> mm(4 * Rn);
    {
        int32_t *dmm = nullptr;
        if ((e = dalloc(c, &dmm, 4 * Rn)) != cudaSuccess) return fail(e);
        k_bminmax<<<Rn, BT, 0, c.stream>>>(b.rels, b.roff, dmm); c.launches++;
        e = cudaMemcpyAsync(mm.data(), dmm, sizeof(int32_t) * 4 * Rn, cudaMemcpyDeviceToHost, c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        cudaFreeAsync(dmm, c.stream);
        if (e != cudaSuccess) return fail(e);
    }
    uint64_t ra = 0, rb = 0;
    int64_t S_cap = 0, dsize = 0;
    for (int i = 0; i < Rn; i++) {
        brel[i].min_a = mm[4 * i];
        brel[i].min_b = mm[4 * i + 2];
        uint64_t rng_a = (uint64_t)((int64_t)mm[4 * i + 1] - (int64_t)mm[4 * i]);
        uint64_t rng_b = (uint64_t)((int64_t)mm[4 * i + 3] - (int64_t)mm[4 * i + 2]);
        ra = std::max(ra, rng_a);
        rb = std::max(rb, rng_b);
        int64_t n = roff[i + 1] - roff[i];
        S_cap += std::min<int64_t>(n, (int64_t)rng_a + 1);
        if (!brel[i].is_root) {
            brel[i].doff = dsize;
            brel[i].range = (uint32_t)(rng_a + 1);
            dsize += (int64_t)rng_a + 1;
        }
    }
    b.bk.bits_a = bits_of(ra);
    b.bk.bits_b = bits_of(rb);
    b.bk.mask_a = b.bk.bits_a ? (~0ull >> (64 - b.bk.bits_a)) : 0;
    b.bk.mask_b = b.bk.bits_b ? (~0ull >> (64 - b.bk.bits_b)) : 0;
    b.key_bits = b.bk.bits_a + b.bk.bits_b + bits_of((uint64_t)std::max(Rn - 1, 0));
    if (b.key_bits > 64) { batch_free(b); if (dev_prev != c.device) cudaSetDevice(dev_prev); return GJ_ERR_INVALID; }
    b.S_cap = std::max<int64_t>(S_cap, 1);
    b.dense_size = dsize;
    if ((e = cudaMemcpyAsync(b.rels, brel.data(), sizeof(BRel) * Rn, cudaMemcpyHostToDevice, c.stream))) return fail(e);
    // tile -> relation of its first row, for the packer
    const int64_t N = b.N;
    std::vector<int32_t> tile_rel(std::max<int64_t>(1, ceil_div(N, PACK_TILE)));
    {
        int r = 0;
        for (int64_t t = 0; t < (int64_t)tile_rel.size(); t++) {
            int64_t row = t * PACK_TILE;
            while (r + 1 < Rn && roff[r + 1] <= row) r++;
            tile_rel[t] = r;
        }
    }
    if ((e = dalloc(c, &b.tile_rel, tile_rel.size())) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(b.tile_rel, tile_rel.data(), sizeof(int32_t) * tile_rel.size(), cudaMemcpyHostToDevice, c.stream))) return fail(e);
    // workspace
    b.status_tiles = std::max<int64_t>(1, ceil_div(N, 4096));
    b.scan_bytes = scan_u32_state_bytes(std::max<int64_t>(N, 1));
    if ((e = dalloc(c, &b.keys, N)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.k2, N)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.ghead, N)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.shead, N)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.gid, N)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.sid, N)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.counts, 4)) != cudaSuccess) return fail(e);
    if ((e = dalloc_bytes(c, &b.scan_state[0], b.scan_bytes)) != cudaSuccess) return fail(e);
    if ((e = dalloc_bytes(c, &b.scan_state[1], b.scan_bytes)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.hist, 8 * 256 + 8)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.status, b.status_tiles * 256)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.gstart, N + 1)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.gsid, N)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.dense, std::max<int64_t>(dsize, 1))) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.rel_gbeg, Rn + 1)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.rel_sbeg, Rn + 1)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.msg_lo, b.S_cap)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.msg_carry, b.S_cap)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.tot_lo, n_queries)) != cudaSuccess) return fail(e);
    if ((e = dalloc(c, &b.tot_carry, n_queries)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(c.stream)) != cudaSuccess) return fail(e);
    if (dev_prev != c.device) cudaSetDevice(dev_prev);
    *out = bb.release();
    return GJ_OK;
}

gj_status gj_batch_set(gj_batch *batch, int32_t param, int64_t value) {
    if (!batch) return GJ_ERR_INVALID;
    if (param == GJ_BATCH_GRID_MULT) {
        if (value < 1 || value > 64) return GJ_ERR_INVALID;
        batch->s.grid_mult = (int)value;
        return GJ_OK;
    }
    return GJ_ERR_INVALID;
}

gj_status gj_batch_info(gj_batch *batch, int64_t *n_rows, int32_t *n_relations, int32_t *levels,
                        int32_t *key_bits) {
    if (!batch) return GJ_ERR_INVALID;
    if (n_rows) *n_rows = batch->s.N;
    if (n_relations) *n_relations = batch->s.R;
    if (levels) *levels = batch->s.levels;
    if (key_bits) *key_bits = batch->s.key_bits;
    return GJ_OK;
}

gj_status gj_batch_run(gj_batch *batch, int32_t use_graph, uint64_t *totals_dev,
                       int32_t *status_dev) {
    if (!batch || !totals_dev) return GJ_ERR_INVALID;
    BatchState &b = batch->s;
    Ctx &c = b.cs->c;
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (dev_prev != c.device) cudaSetDevice(c.device);
    cudaError_t e = cudaSuccess;
    if (b.R == 0) {
        // nothing for the batched kernels
    } else if (!use_graph) {
        e = batch_enqueue(b, c, totals_dev, status_dev);
    } else {
        if (b.exec && (b.g_totals != totals_dev || b.g_status != status_dev || b.g_mult != b.grid_mult)) {
            cudaGraphExecDestroy(b.exec);
            cudaGraphDestroy(b.graph);
            b.exec = nullptr;
            b.graph = nullptr;
        }
        if (!b.exec) {
            if (!b.capture_stream)
                e = cudaStreamCreateWithFlags(&b.capture_stream, cudaStreamNonBlocking);
            Ctx cap = c;
            cap.stream = b.capture_stream;
            cap.launches = 0;
            if (e == cudaSuccess) e = cudaStreamBeginCapture(cap.stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = batch_enqueue(b, cap, totals_dev, status_dev);
                e = cudaStreamEndCapture(cap.stream, &b.graph);
                if (e2 != cudaSuccess) e = e2;
                b.g_launches = cap.launches;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b.exec, b.graph, 0);
            b.g_totals = totals_dev;
            b.g_status = status_dev;
            b.g_mult = b.grid_mult;
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(b.exec, c.stream);
        if (e == cudaSuccess) c.launches += b.g_launches;
    }
    // the other queries, one by one on the same stream (after the batched
    // kernels, which also write their slots), their results copied in
    gj_status st = GJ_OK;
    if (e == cudaSuccess && !b.fallback.empty()) {
        b.fb_total.assign(b.fallback.size(), 0);
        b.fb_status.assign(b.fallback.size(), GJ_OK);
        for (size_t i = 0; i < b.fallback.size() && st == GJ_OK; i++) {
            uint64_t t = 0;
            gj_status s1 = gj_summarize(b.fallback[i].second, &t);
            if (s1 != GJ_OK && s1 != GJ_ERR_OVERFLOW) { st = s1; break; }
            b.fb_total[i] = s1 == GJ_ERR_OVERFLOW ? SAT : t;
            b.fb_status[i] = s1;
        }
        for (size_t i = 0; i < b.fallback.size() && st == GJ_OK && e == cudaSuccess; i++) {
            const int q = b.fallback[i].first;
            e = cudaMemcpyAsync(totals_dev + q, &b.fb_total[i], 8, cudaMemcpyHostToDevice, c.stream);
            if (e == cudaSuccess && status_dev)
                e = cudaMemcpyAsync(status_dev + q, &b.fb_status[i], 4, cudaMemcpyHostToDevice, c.stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);   // the host values are read by then
    }
    if (dev_prev != c.device) cudaSetDevice(dev_prev);
    if (e != cudaSuccess) {
        note_cuda_error(e, __FILE__, __LINE__);
        cudaGetLastError();
        return GJ_ERR_CUDA;
    }
    return st;
}

void gj_batch_destroy(gj_batch *batch) {
    if (!batch) return;
    batch_free(batch->s);
    delete batch;
}

}  // extern "C"
