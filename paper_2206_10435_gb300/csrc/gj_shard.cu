// gj_shard.cu -- one rank's part of the counting pass of a row-sharded query.
//
// When every relation is split by rows across ranks, Algorithm 2 still
// works edge by edge: the message of a relation t to its parent sums, over
// t's rows with separator value v, the product of t's children's messages
// at the row's keys (Eqs. 6-10), and a sum over all rows is the sum over
// the ranks' rows.  So each rank computes a partial message from its own
// groups and the children's *global* messages, the ranks add the partials
// exactly (a saturating sum), and the result is the global message the
// parent's ranks use.  The root's partials add up to |Q|.  The downward
// pass mirrors it: with t's global down message, each rank's partial down
// messages to t's children, added over the ranks.  A group's multiplicity
// (its marginal over the result, Section 1.2) is w (x) down; on a rank it
// covers the rank's rows of that key tuple, and the ranks' values for one
// key tuple add up to the global one.
//
// Messages here are dense vectors over the separator attribute's value
// domain [lo, lo + len), which every rank uses alike (the caller agrees on
// it from gj_shard_domain's local ranges).  Partial sums are accumulated
// exactly: the 32-bit halves of each contribution are added with
// non-returning 64-bit atomics (fewer than 2^31 contributions, so neither
// wraps) and a flag marks a saturated contribution.
#include <algorithm>

#include "gj_state.cuh"

namespace gj {
namespace {

constexpr int SH = 256;

struct Acc {
    unsigned long long *lo, *hi;
    unsigned int *sat;
};

struct ShardSpec {
    int64_t G;
    const uint32_t *gstart;
    int root;
    const int32_t *skey;              // the relation's separator column (by group)
    int nch;
    const int32_t *ckey[MAX_REL];     // its column holding child c's separator value
    const uint64_t *cmsg[MAX_REL];    // child c's global message
    int32_t clo[MAX_REL];
    int64_t clen[MAX_REL];
    // upward: the partial message (or the root's partial total at 0)
    Acc up;
    int32_t lo;
    int64_t len;
    // downward: the relation's global down message, children's partials
    const uint64_t *down;
    int32_t dlo;
    int64_t dlen;
    Acc cdown[MAX_REL];
    uint64_t *mult;
    uint32_t *err;
};

__device__ __forceinline__ uint64_t dense_at(const uint64_t *m, int32_t lo, int64_t len, int32_t key) {
    const int64_t d = (int64_t)key - (int64_t)lo;
    return (d >= 0 && d < len) ? __ldg((const unsigned long long *)m + d) : 0ull;
}

__device__ __forceinline__ void acc_add(const Acc &a, int64_t i, uint64_t x) {
    if (x == 0) return;
    if (x == SAT) { atomicOr(a.sat + i, 1u); return; }
    atomicAdd(a.lo + i, (unsigned long long)(x & 0xffffffffull));
    if (x >> 32) atomicAdd(a.hi + i, (unsigned long long)(x >> 32));
}

__global__ void k_shard_up(ShardSpec s) {
    for (int64_t g = (int64_t)blockIdx.x * SH + threadIdx.x; g < s.G; g += (int64_t)gridDim.x * SH) {
        uint64_t w = (uint64_t)(s.gstart[g + 1] - s.gstart[g]);
        for (int c = 0; c < s.nch && w; c++)
            w = sat_mul(w, dense_at(s.cmsg[c], s.clo[c], s.clen[c], s.ckey[c][g]));
        int64_t i = 0;
        if (!s.root) {
            i = (int64_t)s.skey[g] - (int64_t)s.lo;
            if (i < 0 || i >= s.len) { raise_err(s.err, ERRF_BOUNDS); continue; }
        }
        acc_add(s.up, i, w);
    }
}

__global__ void k_shard_down(ShardSpec s) {
    for (int64_t g = (int64_t)blockIdx.x * SH + threadIdx.x; g < s.G; g += (int64_t)gridDim.x * SH) {
        const uint64_t cnt = (uint64_t)(s.gstart[g + 1] - s.gstart[g]);
        const uint64_t d = s.root ? 1ull : dense_at(s.down, s.dlo, s.dlen, s.skey[g]);
        uint64_t w = cnt;
        for (int c = 0; c < s.nch; c++) w = sat_mul(w, dense_at(s.cmsg[c], s.clo[c], s.clen[c], s.ckey[c][g]));
        s.mult[g] = sat_mul(w, d);
        const uint64_t base = sat_mul(cnt, d);
        if (base == 0) continue;
        for (int c = 0; c < s.nch; c++) {
            uint64_t x = base;
            for (int o = 0; o < s.nch && x; o++)
                if (o != c) x = sat_mul(x, dense_at(s.cmsg[o], s.clo[o], s.clen[o], s.ckey[o][g]));
            const int64_t i = (int64_t)s.ckey[c][g] - (int64_t)s.clo[c];
            if (i < 0 || i >= s.clen[c]) continue;   // no rank holds that value in the child
            acc_add(s.cdown[c], i, x);
        }
    }
}

// out[i] = hi * 2^32 + lo, saturated at SAT
__global__ void k_acc_finish(Acc a, int64_t len, uint64_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * SH + threadIdx.x; i < len; i += (int64_t)gridDim.x * SH) {
        if (a.sat[i]) { out[i] = SAT; continue; }
        const uint64_t lo = a.lo[i], top = a.hi[i] + (lo >> 32);
        if (top >> 32) { out[i] = SAT; continue; }
        const uint64_t v = (top << 32) | (lo & 0xffffffffull);
        out[i] = v == SAT ? SAT : v;
    }
}

inline int grid_of(Ctx &c, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, SH), (int64_t)c.num_sms * 16));
}

cudaError_t acc_alloc(Ctx &c, Acc &a, int64_t len, void **mem) {
    const size_t n = (size_t)std::max<int64_t>(len, 1);
    GJ_CUDA_TRY(dalloc_bytes(c, mem, n * 20));
    GJ_CUDA_TRY(cudaMemsetAsync(*mem, 0, n * 20, c.stream));
    a.lo = (unsigned long long *)*mem;
    a.hi = a.lo + n;
    a.sat = (unsigned int *)(a.hi + n);
    return cudaSuccess;
}

// The query's tree around relation rel, for the sharded pass: every
// separator must be one attribute.
bool shard_spec(QueryState &q, int rel, ShardSpec &s) {
    s = ShardSpec{};
    if (q.tri || q.cyc || rel < 0 || rel >= q.k) return false;
    QRel &t = q.r[rel];
    if (t.parent >= 0 && t.sep_cols.size() != 1) return false;
    s.G = t.F->G;
    s.gstart = t.F->gstart;
    s.root = t.parent < 0;
    if (!s.root) s.skey = t.F->gkey + (int64_t)t.sep_cols[0] * t.F->G;
    s.nch = (int)t.children.size();
    for (int ci = 0; ci < s.nch; ci++) {
        const QRel &ch = q.r[t.children[ci]];
        if (ch.sep_cols_parent.size() != 1) return false;
        s.ckey[ci] = t.F->gkey + (int64_t)ch.sep_cols_parent[0] * t.F->G;
    }
    s.err = q.ctx().err;
    return true;
}

gj_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return GJ_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
}

}  // namespace

gj_status check_device_error(Ctx &c);

}  // namespace gj

using namespace gj;

extern "C" {

gj_status gj_shard_domain(gj_query *q, int32_t rel, int32_t *lo, int32_t *hi) {
    if (!q || !lo || !hi) return GJ_ERR_INVALID;
    QueryState &s = q->s;
    if (s.tri || s.cyc || rel < 0 || rel >= s.k || s.r[rel].parent < 0) return GJ_ERR_INVALID;
    const QRel &t = s.r[rel];
    if (t.sep_cols.size() != 1 || t.sep_cols_parent.size() != 1) return GJ_ERR_INVALID;
    const QRel &p = s.r[t.parent];
    int32_t a = INT32_MAX, b = INT32_MIN;
    if (t.R->n > 0) { a = std::min(a, t.R->kmin[t.sep_cols[0]]); b = std::max(b, t.R->kmax[t.sep_cols[0]]); }
    if (p.R->n > 0) {
        a = std::min(a, p.R->kmin[t.sep_cols_parent[0]]);
        b = std::max(b, p.R->kmax[t.sep_cols_parent[0]]);
    }
    *lo = a;
    *hi = b;   // empty on this rank when lo > hi
    return GJ_OK;
}

gj_status gj_shard_up(gj_query *q, int32_t rel, const uint64_t *const *child_msg, const int32_t *child_lo,
                      const int64_t *child_len, uint64_t *msg_out, int32_t lo, int64_t len) {
    if (!q || !msg_out) return GJ_ERR_INVALID;
    QueryState &s = q->s;
    ShardSpec sp;
    if (!shard_spec(s, rel, sp)) return GJ_ERR_INVALID;
    if (sp.nch && (!child_msg || !child_lo || !child_len)) return GJ_ERR_INVALID;
    if (sp.root) { lo = 0; len = 1; }
    if (len < 1) return GJ_ERR_INVALID;
    for (int c = 0; c < sp.nch; c++) {
        if (child_len[c] < 0 || (child_len[c] > 0 && !child_msg[c])) return GJ_ERR_INVALID;
        sp.cmsg[c] = child_msg[c];
        sp.clo[c] = child_lo[c];
        sp.clen[c] = child_len[c];
    }
    sp.lo = lo;
    sp.len = len;
    Ctx &c = s.ctx();
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != s.cs->c.device) cudaSetDevice(s.cs->c.device);
    void *mem = nullptr;
    cudaError_t e = acc_alloc(c, sp.up, len, &mem);
    if (e == cudaSuccess && sp.G > 0) {
        k_shard_up<<<grid_of(c, sp.G), SH, 0, c.stream>>>(sp); c.launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_acc_finish<<<grid_of(c, len), SH, 0, c.stream>>>(sp.up, len, msg_out); c.launches++;
        e = cudaGetLastError();
    }
    dfree(c, mem);
    gj_status st = status_of(e);
    if (st == GJ_OK) st = check_device_error(c);
    if (dev != s.cs->c.device) cudaSetDevice(dev);
    return st;
}

gj_status gj_shard_down(gj_query *q, int32_t rel, const uint64_t *down_in, int32_t down_lo, int64_t down_len,
                        const uint64_t *const *child_msg, const int32_t *child_lo,
                        const int64_t *child_len, uint64_t *const *child_down_out, uint64_t *mult_out) {
    if (!q || !mult_out) return GJ_ERR_INVALID;
    QueryState &s = q->s;
    ShardSpec sp;
    if (!shard_spec(s, rel, sp)) return GJ_ERR_INVALID;
    if (!sp.root && (!down_in || down_len < 1)) return GJ_ERR_INVALID;
    if (sp.nch && (!child_msg || !child_lo || !child_len || !child_down_out)) return GJ_ERR_INVALID;
    for (int c = 0; c < sp.nch; c++) {
        if (child_len[c] < 1 || !child_msg[c] || !child_down_out[c]) return GJ_ERR_INVALID;
        sp.cmsg[c] = child_msg[c];
        sp.clo[c] = child_lo[c];
        sp.clen[c] = child_len[c];
    }
    sp.down = down_in;
    sp.dlo = down_lo;
    sp.dlen = down_len;
    sp.mult = mult_out;
    Ctx &c = s.ctx();
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != s.cs->c.device) cudaSetDevice(s.cs->c.device);
    std::vector<void *> mem(sp.nch, nullptr);
    cudaError_t e = cudaSuccess;
    for (int ci = 0; ci < sp.nch && e == cudaSuccess; ci++) e = acc_alloc(c, sp.cdown[ci], sp.clen[ci], &mem[ci]);
    if (e == cudaSuccess && sp.G > 0) {
        k_shard_down<<<grid_of(c, sp.G), SH, 0, c.stream>>>(sp); c.launches++;
        e = cudaGetLastError();
    }
    for (int ci = 0; ci < sp.nch && e == cudaSuccess; ci++) {
        k_acc_finish<<<grid_of(c, sp.clen[ci]), SH, 0, c.stream>>>(sp.cdown[ci], sp.clen[ci], child_down_out[ci]); c.launches++;
        e = cudaGetLastError();
    }
    for (void *&m : mem) dfree(c, m);
    gj_status st = status_of(e);
    if (st == GJ_OK) st = check_device_error(c);
    if (dev != s.cs->c.device) cudaSetDevice(dev);
    return st;
}

}  // extern "C"
