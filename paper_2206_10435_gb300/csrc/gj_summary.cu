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
//
// Kernels.  Per relation, the whole upward step is one single-pass scan
// (decoupled lookback) whose element is (w, live, head): w computed from the
// counts and the children's messages, head marking the first group of a
// separator segment, live = w > 0.  Its combine is a segmented saturating sum
// of w next to plain counts of heads and live groups, so one pass yields the
// in-segment offsets, the messages (segment sums), the segment numbering
// and the compaction of the live groups the desummariser walks.  Per
// relation, the downward step is one kernel: mult, and every child's down
// message accumulated exactly by non-returning 64-bit atomic adds of the
// contributions' 32-bit halves (the true sum is recovered in 128 bits, so
// saturation is exact).
#include <algorithm>
#include <atomic>

#include "gj_lookback.cuh"
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

inline int grid_for(Ctx &c, int64_t n) {
    int64_t b = ceil_div(n, ST);
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)c.num_sms * 16));
}

#define GRID_LOOP(i, n) \
    for (int64_t i = (int64_t)blockIdx.x * ST + threadIdx.x; i < (n); i += (int64_t)gridDim.x * ST)

__global__ void k_fill_u32(uint32_t *p, int64_t n, uint32_t v) {
    GRID_LOOP(i, n) p[i] = v;
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

// ------------------------------------------------------------ upward scan
// Scan state of a run of groups: v = saturating sum of w since the last
// segment head (inclusive of everything when there is none), nh = heads,
// nl = live groups.  (a) . (b) = (b.nh ? b.v : a.v (+) b.v, a.nh + b.nh,
// a.nl + b.nl): associative, not commutative.
struct UpState {
    uint64_t v;
    uint32_t nh, nl;
};

__device__ __forceinline__ UpState up_op(const UpState &a, const UpState &b) {
    UpState r;
    r.v = b.nh ? b.v : sat_add(a.v, b.v);
    r.nh = a.nh + b.nh;
    r.nl = a.nl + b.nl;
    return r;
}

__device__ __forceinline__ UpState up_shfl_up(const UpState &x, int d) {
    UpState r;
    r.v = __shfl_up_sync(0xffffffffu, x.v, d);
    r.nh = __shfl_up_sync(0xffffffffu, x.nh, d);
    r.nl = __shfl_up_sync(0xffffffffu, x.nl, d);
    return r;
}

__device__ __forceinline__ UpState up_shfl_down(const UpState &x, int d) {
    UpState r;
    r.v = __shfl_down_sync(0xffffffffu, x.v, d);
    r.nh = __shfl_down_sync(0xffffffffu, x.nh, d);
    r.nl = __shfl_down_sync(0xffffffffu, x.nl, d);
    return r;
}

__device__ __forceinline__ UpState up_shfl(const UpState &x, int l) {
    UpState r;
    r.v = __shfl_sync(0xffffffffu, x.v, l);
    r.nh = __shfl_sync(0xffffffffu, x.nh, l);
    r.nl = __shfl_sync(0xffffffffu, x.nl, l);
    return r;
}

// A tile's published state: flag, heads and live count in one word (the
// counts are below 2^31), the sum in the other, moved as one 16-byte access.
__device__ __forceinline__ void up_put(ulonglong2 *s, uint32_t f, const UpState &x) {
    const unsigned long long a = (unsigned long long)f | ((unsigned long long)x.nh << 2) |
                                 ((unsigned long long)x.nl << 33);
    asm volatile("st.volatile.global.v2.u64 [%0], {%1, %2};" ::"l"(s), "l"(a),
                 "l"((unsigned long long)x.v)
                 : "memory");
}

__device__ __forceinline__ void up_get(const ulonglong2 *s, uint32_t &f, UpState &x) {
    unsigned long long a, b;
    asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(s) : "memory");
    f = (uint32_t)(a & 3u);
    x.nh = (uint32_t)((a >> 2) & 0x7fffffffu);
    x.nl = (uint32_t)(a >> 33);
    x.v = b;
}

// Decoupled lookback by one warp for the ordered (non-commutative) combine:
// the window of 32 predecessors is folded in tile order by a shuffle-down
// tree.  Polls are bounded by SPIN_LIMIT (ERRF_TIMEOUT on expiry, the
// predecessor then counts as an empty prefix).
__device__ UpState up_lookback(ulonglong2 *st, uint32_t tile, const UpState &agg, int lane,
                               uint32_t *err) {
    const UpState zero{0ull, 0u, 0u};
    if (tile == 0) {
        if (lane == 0) up_put(&st[0], ST_P, agg);
        return zero;
    }
    if (lane == 0) up_put(&st[tile], ST_A, agg);
    UpState carry = zero;
    int64_t p = (int64_t)tile - 1;
    for (;;) {
        const int64_t q = p - 31 + lane;
        uint32_t f = ST_P;
        UpState v = zero;
        if (q >= 0) {
            uint32_t spins = 0;
            for (;;) {
                up_get(&st[q], f, v);
                if (f) break;
                if (++spins > SPIN_LIMIT) {
                    raise_err(err, ERRF_TIMEOUT);
                    f = ST_P;
                    v = zero;
                    break;
                }
            }
        }
        const uint32_t pm = __ballot_sync(0xffffffffu, f == ST_P);
        const int hi = pm ? 31 - __clz((int)pm) : 0;
        UpState x = lane >= hi ? v : zero;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const UpState y = up_shfl_down(x, d);
            if (lane + d < 32) x = up_op(x, y);
        }
        x = up_shfl(x, 0);
        carry = up_op(x, carry);
        if (pm) break;
        p -= 32;
    }
    if (lane == 0) up_put(&st[tile], ST_P, up_op(carry, agg));
    return carry;
}

struct UpSpec {
    int64_t G;
    const uint32_t *gstart;            // counts: gstart[g + 1] - gstart[g]
    int nch;
    const uint32_t *link[MAX_REL];     // children's links and messages
    const uint64_t *msg[MAX_REL];
    int seg;                           // segmented by the separator (non-root)
    KeyCols sep;                       // separator key columns (heads)
    // outputs
    uint64_t *w, *off;
    uint64_t *msg_out;                 // [S] segment sums (non-root)
    uint32_t *seg_id, *seg_first;      // [G], [S+1] (non-root)
    uint32_t *S_dev;
    uint32_t *lgid;                    // live groups: [L]
    uint64_t *loff, *lw;
    uint32_t *lseg_first;              // [S+1] (non-root)
    uint32_t *L_dev;
    uint64_t *total;                   // root: sum of all w
    // dense link table of this relation's segments (one separator column of
    // small range): dense[key - dense_mn] = segment
    uint32_t *dense;
    const int32_t *dense_key;
    int32_t dense_mn;
    // lookback
    ulonglong2 *status;
    uint32_t *counter;
    uint32_t *err;
};

constexpr int UP_ITEMS = 8;
constexpr int UP_TILE = ST * UP_ITEMS;

// shared-memory slot of element e: one pad slot per 16 (64-bit arrays) or
// 32 (32-bit arrays) elements keeps both the coalesced (warp on 32
// consecutive elements) and the per-thread (thread on UP_ITEMS consecutive
// elements) phases free of bank conflicts
__device__ __forceinline__ int p64(int e) { return e + (e >> 4); }
__device__ __forceinline__ int p32(int e) { return e + (e >> 5); }
constexpr int UP_S64 = UP_TILE + UP_TILE / 16;
constexpr int UP_S32 = UP_TILE + UP_TILE / 32;
constexpr size_t UP_SMEM = 2 * (size_t)UP_S64 * 8 + 2 * (size_t)UP_S32 * 4 + UP_TILE;

__device__ __forceinline__ bool sep_head(const KeyCols &sep, int64_t g) {
    if (g == 0) return true;
    for (int c = 0; c < sep.ncol; c++)
        if (__ldg(sep.col[c] + g) != __ldg(sep.col[c] + g - 1)) return true;
    return false;
}

// NCH >= 0: exactly NCH children; NCH < 0: s.nch.  SEP1: the separator is
// one column (heads found from a staged copy of it), else any number.
template <int NCH, bool SEP1>
__global__ void __launch_bounds__(ST, NCH >= 3 ? 3 : 1)
k_up_scan(UpSpec s) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *s_w = (uint64_t *)smem;                 // the element's w
    uint64_t *s_xv = s_w + UP_S64;                    // exclusive v
    uint32_t *s_xh = (uint32_t *)(s_xv + UP_S64);     // exclusive heads
    uint32_t *s_xl = s_xh + UP_S32;                   // exclusive live groups
    uint8_t *s_h = (uint8_t *)(s_xl + UP_S32);        // head flag
    __shared__ UpState s_warp[ST / 32];
    __shared__ UpState s_carry;
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(s.counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * UP_TILE;
    if (base >= s.G) return;
    const int tile_n = (int)min((int64_t)UP_TILE, s.G - base);
    // elements, coalesced (element e = tid + i * ST): every independent load
    // of the tile is issued before the first use -- group starts, separator
    // keys, the children's links -- then the messages behind the links
    uint32_t *s_gs = s_xh;              // group starts [0, tile_n]; s_xh is free until the scan
    int32_t *s_key = (int32_t *)s_xl;   // separator key of element e at e + 1; [0] the one before
    const int nch = NCH >= 0 ? NCH : s.nch;
    uint32_t gs[UP_ITEMS];
    int32_t key[UP_ITEMS];
    uint64_t prod[UP_ITEMS];
#pragma unroll
    for (int i = 0; i < UP_ITEMS; i++) {
        const int e = tid + i * ST;
        const bool in = e < tile_n;
        gs[i] = in ? __ldg(s.gstart + base + e) : 0u;
        if (SEP1) key[i] = in && s.seg ? __ldg(s.sep.col[0] + base + e) : 0;
        prod[i] = 1;
    }
    if (tid == 0) {
        s_gs[tile_n] = __ldg(s.gstart + base + tile_n);
        if (SEP1) s_key[0] = base > 0 && s.seg ? __ldg(s.sep.col[0] + base - 1) : 0;
    }
#pragma unroll
    for (int c = 0; c < (NCH >= 0 ? NCH : MAX_REL); c++) {
        if (NCH < 0 && c >= nch) break;
        const uint32_t *lk = s.link[c];
        const unsigned long long *mg = (const unsigned long long *)s.msg[c];
        uint32_t l[UP_ITEMS];
#pragma unroll
        for (int i = 0; i < UP_ITEMS; i++) {
            const int e = tid + i * ST;
            l[i] = e < tile_n ? __ldg(lk + base + e) : NONE;
        }
#pragma unroll
        for (int i = 0; i < UP_ITEMS; i++)
            prod[i] = sat_mul(prod[i], l[i] == NONE ? 0ull : __ldg(mg + l[i]));
    }
#pragma unroll
    for (int i = 0; i < UP_ITEMS; i++) {
        const int e = tid + i * ST;
        if (e < tile_n) s_gs[e] = gs[i];   // [tile_n] is thread 0's
        if (SEP1) s_key[e + 1] = key[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < UP_ITEMS; i++) {
        const int e = tid + i * ST;
        uint64_t w = 0;
        uint8_t h = 0;
        if (e < tile_n) {
            // w = cnt (x) prod of the children's messages (the semiring
            // product is associative and commutative)
            w = sat_mul((uint64_t)(s_gs[e + 1] - s_gs[e]), prod[i]);
            if (s.seg) {
                if (SEP1) h = (base + e == 0) || s_key[e + 1] != s_key[e];
                else h = sep_head(s.sep, base + e);
            }
        }
        s_w[p64(e)] = w;
        s_h[e] = h;
    }
    __syncthreads();
    // each thread: UP_ITEMS consecutive elements
    UpState run{0ull, 0u, 0u};
#pragma unroll
    for (int i = 0; i < UP_ITEMS; i++) {
        const int e = tid * UP_ITEMS + i;
        const UpState x{s_w[p64(e)], (uint32_t)s_h[e], s_w[p64(e)] != 0 ? 1u : 0u};
        run = up_op(run, x);
    }
    // warp inclusive scan of the threads' states, in order
    UpState inc = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const UpState y = up_shfl_up(inc, d);
        if (lane >= d) inc = up_op(y, inc);
    }
    if (lane == 31) s_warp[warp] = inc;
    UpState ex = up_shfl_up(inc, 1);
    if (lane == 0) ex = UpState{0ull, 0u, 0u};
    __syncthreads();
    UpState before{0ull, 0u, 0u};
    for (int w = 0; w < warp; w++) before = up_op(before, s_warp[w]);
    if (warp == ST / 32 - 1) {
        // the tile's aggregate (last warp), then its carry-in
        UpState agg{0ull, 0u, 0u};
        for (int w = 0; w < ST / 32; w++) agg = up_op(agg, s_warp[w]);
        const UpState carry = up_lookback(s.status, tile, agg, lane, s.err);
        if (lane == 0) {
            s_carry = carry;
            if (base + UP_TILE >= s.G) {   // the last tile: totals
                const UpState all = up_op(carry, agg);
                if (s.seg) {
                    *s.S_dev = all.nh;
                    s.seg_first[all.nh] = (uint32_t)s.G;
                    s.lseg_first[all.nh] = all.nl;
                } else if (s.total) {
                    *s.total = all.v;
                }
                *s.L_dev = all.nl;
            }
        }
    }
    __syncthreads();
    // exclusive state of each of the thread's elements
    UpState x = up_op(up_op(s_carry, before), ex);
#pragma unroll
    for (int i = 0; i < UP_ITEMS; i++) {
        const int e = tid * UP_ITEMS + i;
        s_xv[p64(e)] = x.v;
        s_xh[p32(e)] = x.nh;
        s_xl[p32(e)] = x.nl;
        const UpState y{s_w[p64(e)], (uint32_t)s_h[e], s_w[p64(e)] != 0 ? 1u : 0u};
        x = up_op(x, y);
    }
    __syncthreads();
    // outputs, coalesced
    for (int e = tid; e < tile_n; e += ST) {
        const int64_t g = base + e;
        const uint64_t w = s_w[p64(e)];
        const bool h = s_h[e] != 0;
        const uint64_t xv = s_xv[p64(e)];
        const uint32_t xl = s_xl[p32(e)];
        const uint64_t off = h ? 0ull : xv;
        s.w[g] = w;
        s.off[g] = off;
        if (s.seg) {
            const uint32_t sid = s_xh[p32(e)] + (h ? 1u : 0u) - 1u;
            s.seg_id[g] = sid;
            if (h) {
                s.seg_first[sid] = (uint32_t)g;
                s.lseg_first[sid] = xl;
                if (s.dense) s.dense[(uint32_t)__ldg(s.dense_key + g) - (uint32_t)s.dense_mn] = sid;
            }
            // the segment's last group writes its message
            const bool last = (g + 1 == s.G) || (e + 1 < tile_n ? s_h[e + 1] != 0 : sep_head(s.sep, g + 1));
            if (last) s.msg_out[sid] = sat_add(off, w);
        }
        if (w != 0) {
            s.lgid[xl] = (uint32_t)g;
            s.loff[xl] = off;
            s.lw[xl] = w;
        }
    }
}

template <int NCH, bool SEP1>
cudaError_t launch_up_scan_k(Ctx &c, const UpSpec &u) {
    // the shared-memory limit is set once per device (devices 0..63)
    static std::atomic<uint64_t> set_on{0};
    const uint64_t bit = 1ull << (c.device & 63);
    if (!(set_on.load(std::memory_order_acquire) & bit)) {
        cudaError_t e = cudaFuncSetAttribute(k_up_scan<NCH, SEP1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)UP_SMEM);
        if (e != cudaSuccess) return e;
        set_on.fetch_or(bit, std::memory_order_release);
    }
    k_up_scan<NCH, SEP1><<<(unsigned)ceil_div(u.G, UP_TILE), ST, UP_SMEM, c.stream>>>(u);
    c.launches++;
    return cudaGetLastError();
}

template <bool SEP1>
cudaError_t launch_up_scan_t(Ctx &c, const UpSpec &u) {
    switch (u.nch) {
        case 0: return launch_up_scan_k<0, SEP1>(c, u);
        case 1: return launch_up_scan_k<1, SEP1>(c, u);
        case 2: return launch_up_scan_k<2, SEP1>(c, u);
        case 3: return launch_up_scan_k<3, SEP1>(c, u);
        case 4: return launch_up_scan_k<4, SEP1>(c, u);
        default: return launch_up_scan_k<-1, SEP1>(c, u);
    }
}

cudaError_t launch_up_scan(Ctx &c, const UpSpec &u) {
    return (!u.seg || u.sep.ncol == 1) ? launch_up_scan_t<true>(c, u) : launch_up_scan_t<false>(c, u);
}

// ------------------------------------------------------------ downward
// A child's down message, accumulated exactly: lo = sum of the
// contributions' low 32-bit halves, hi = sum of their high halves (fewer
// than 2^31 contributions, so neither wraps), sat = a contribution was
// SAT.  The value is hi * 2^32 + lo, saturated at SAT.
struct DownAcc {
    unsigned long long *lo, *hi;
    unsigned int *sat;
};

__device__ __forceinline__ uint64_t down_value(const DownAcc &a, uint32_t s) {
    if (a.sat[s]) return SAT;
    const uint64_t lo = a.lo[s], hi = a.hi[s];
    const uint64_t top = hi + (lo >> 32);
    if (top >> 32) return SAT;
    const uint64_t v = (top << 32) | (lo & 0xffffffffull);
    return v == SAT ? SAT : v;
}

struct DownSpec {
    int64_t G;
    const uint32_t *gstart;
    const uint64_t *w;
    uint64_t *mult;
    // this relation's own down message (non-root)
    int has_down;
    DownAcc self;
    const uint32_t *seg_id, *seg_first;
    uint64_t *down_out;                // [S] the finished values
    // children
    int nch;
    const uint32_t *link[MAX_REL];
    const uint64_t *msg[MAX_REL];
    DownAcc acc[MAX_REL];
    uint8_t agg[MAX_REL];              // combine child c's contributions per block
};

// Contributions to a child's down message are combined per block before
// they reach global memory when the parent's links to that child are not in
// key order: parent groups of skewed keys send many contributions to the
// same child segment (on a Zipf(1.1) chain, 3.6% of a relation's groups
// link to its most common key), and atomics on one address serialise.
// Each round a block accumulates contributions in a small open-addressing
// table in shared memory, segment -> 16-bit pieces of the sum (32-bit
// counters: a round adds at most ST * DN_ITEMS pieces below 2^16, so none
// wraps) and a SAT flag; once the table is full, contributions of new
// segments go to the global accumulators directly.  A key that recurs in a
// round (the hot ones) claims a slot early and is added once per round
// and block.  At the end of the round every claimed slot is added to the
// global split-word accumulators.  Integer sums: exact in any order.
// Links in key order (the child joins the parent's leading columns) go
// straight to the global accumulators.  A block also stops using the table
// for a child while fewer than one in AGG_MIN_HIT of a round's
// contributions find their key already there (keys without repeats: the
// table would only add work), and tries it again every AGG_RETRY rounds.
constexpr int AGG_BITS = 8;
constexpr int AGG = 1 << AGG_BITS;
constexpr int AGG_PROBES = 2;
constexpr uint32_t AGG_MIN_HIT = 16;
constexpr int AGG_RETRY = 8;

struct AggTable {
    uint32_t key[AGG];
    uint32_t piece[4][AGG];   // the sum's bits [16 p, 16 p + 16), p = 0..3, summed
    uint32_t sat[AGG];
};

__device__ __forceinline__ void acc_add_global(const DownAcc &a, uint32_t l, uint64_t x) {
    if (x == SAT) {
        atomicOr(a.sat + l, 1u);
        return;
    }
    // results unused: compiled to fire-and-forget reductions
    atomicAdd(a.lo + l, (unsigned long long)(x & 0xffffffffull));
    if (x >> 32) atomicAdd(a.hi + l, (unsigned long long)(x >> 32));
}

// Returns 1 when l already had a slot (a repeated key).
__device__ __forceinline__ uint32_t agg_add(AggTable &t, const DownAcc &a, uint32_t l, uint64_t x) {
    uint32_t slot = (l * 0x9E3779B1u) >> (32 - AGG_BITS);
#pragma unroll
    for (int p = 0; p < AGG_PROBES; p++) {
        uint32_t k = *(volatile uint32_t *)(t.key + slot);
        if (k == NONE) k = atomicCAS(t.key + slot, NONE, l);   // the old value: NONE = claimed now
        if (k == NONE || k == l) {
            if (x == SAT) {
                atomicOr(t.sat + slot, 1u);
            } else {
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t v = (uint32_t)(x >> (16 * q)) & 0xffffu;
                    if (v) atomicAdd(&t.piece[q][slot], v);
                }
            }
            return k == l ? 1u : 0u;
        }
        slot = (slot + 1) & (AGG - 1);
    }
    acc_add_global(a, l, x);
    return 0;
}

// NCH >= 0: exactly NCH children, DN_ITEMS groups per thread and round with
// every independent load issued before the first use, contributions
// combined per block (dynamic shared memory AGG_SMEM when NCH > 0);
// NCH < 0: s.nch children, one group per thread and round, contributions
// straight to the global accumulators
constexpr int DN_ITEMS = 4;

template <int NCH>
__global__ void __launch_bounds__(ST)
k_down(DownSpec s) {
    constexpr int CAP = NCH >= 0 ? (NCH > 0 ? NCH : 1) : MAX_REL;
    constexpr int IT = NCH >= 3 ? DN_ITEMS / 2 : NCH >= 0 ? DN_ITEMS : 1;   // fewer registers with many children
    const int nch = NCH >= 0 ? NCH : s.nch;
    __shared__ AggTable tab;
    __shared__ uint32_t s_use[CAP], s_hits[CAP];
    if (NCH > 0 && threadIdx.x < CAP) s_use[threadIdx.x] = 1;   // seen after the first barrier
    const int64_t step = (int64_t)gridDim.x * ST * IT;
    // b0 is the same for every thread of the block: the rounds (and the
    // barriers in them) are uniform
    int round = 0;
    for (int64_t b0 = (int64_t)blockIdx.x * ST * IT; b0 < s.G; b0 += step, round++) {
        int64_t g[IT];
        bool in[IT];
        uint32_t g0[IT], g1[IT], sid[IT];
        uint64_t w[IT];
#pragma unroll
        for (int i = 0; i < IT; i++) {
            g[i] = b0 + threadIdx.x + (int64_t)i * ST;
            in[i] = g[i] < s.G;
            g0[i] = in[i] ? __ldg(s.gstart + g[i]) : 0u;
            g1[i] = in[i] ? __ldg(s.gstart + g[i] + 1) : 0u;
            w[i] = in[i] ? __ldg((const unsigned long long *)s.w + g[i]) : 0ull;
            sid[i] = in[i] && s.has_down ? __ldg(s.seg_id + g[i]) : 0u;
        }
        uint32_t l[CAP][IT];
        if constexpr (NCH != 0) {
#pragma unroll
            for (int c = 0; c < CAP; c++) {
                if (c >= nch) break;
#pragma unroll
                for (int i = 0; i < IT; i++) l[c][i] = in[i] ? __ldg(s.link[c] + g[i]) : NONE;
            }
        }
        uint64_t d[IT];
        uint32_t first[IT];
#pragma unroll
        for (int i = 0; i < IT; i++) {
            d[i] = 1;
            first[i] = NONE;
            if (in[i] && s.has_down) {
                d[i] = down_value(s.self, sid[i]);
                first[i] = __ldg(s.seg_first + sid[i]);
            }
        }
        uint64_t m[CAP][IT];
        if constexpr (NCH != 0) {
#pragma unroll
            for (int c = 0; c < CAP; c++) {
                if (c >= nch) break;
#pragma unroll
                for (int i = 0; i < IT; i++)
                    m[c][i] = l[c][i] == NONE ? 0ull : __ldg((const unsigned long long *)s.msg[c] + l[c][i]);
            }
        }
        // mult, the relation's own down message; base = cnt (x) down
        uint64_t base[IT];
#pragma unroll
        for (int i = 0; i < IT; i++) {
            base[i] = 0;
            if (!in[i]) continue;
            base[i] = (uint64_t)(g1[i] - g0[i]);
            if (s.has_down) {
                if (first[i] == (uint32_t)g[i]) s.down_out[sid[i]] = d[i];
                base[i] = sat_mul(base[i], d[i]);
                s.mult[g[i]] = sat_mul(w[i], d[i]);
            } else {
                s.mult[g[i]] = w[i];
            }
        }
        if constexpr (NCH > 0) {
            // child c's contributions: base (x) the other children's messages
#pragma unroll
            for (int c = 0; c < NCH; c++) {
                uint64_t x[IT];
#pragma unroll
                for (int i = 0; i < IT; i++) {
                    x[i] = l[c][i] == NONE ? 0ull : base[i];
#pragma unroll
                    for (int j = 0; j < NCH; j++)
                        if (j != c) x[i] = sat_mul(x[i], m[j][i]);
                }
                bool use = s.agg[c] != 0;   // the same for the whole grid
                if (use) {
                    __syncthreads();   // the table's previous use is over; s_use is settled
                    use = s_use[c] || round % AGG_RETRY == 0;   // the same for the block
                }
                if (!use) {
#pragma unroll
                    for (int i = 0; i < IT; i++)
                        if (x[i]) acc_add_global(s.acc[c], l[c][i], x[i]);
                    continue;
                }
                for (int j = threadIdx.x; j < AGG; j += ST) {
                    tab.key[j] = NONE;
                    tab.piece[0][j] = tab.piece[1][j] = tab.piece[2][j] = tab.piece[3][j] = 0;
                    tab.sat[j] = 0;
                }
                if (threadIdx.x == 0) s_hits[c] = 0;
                __syncthreads();
                uint32_t hits = 0;
#pragma unroll
                for (int i = 0; i < IT; i++)
                    if (x[i]) hits += agg_add(tab, s.acc[c], l[c][i], x[i]);
                hits = __reduce_add_sync(0xffffffffu, hits);
                if ((threadIdx.x & 31) == 0 && hits) atomicAdd(&s_hits[c], hits);
                __syncthreads();
                if (threadIdx.x == 0) s_use[c] = s_hits[c] * AGG_MIN_HIT >= (uint32_t)(ST * IT);
                for (int j = threadIdx.x; j < AGG; j += ST) {
                    const uint32_t k = tab.key[j];
                    if (k == NONE) continue;
                    if (tab.sat[j]) atomicOr(s.acc[c].sat + k, 1u);
                    const unsigned long long lo = (unsigned long long)tab.piece[0][j] +
                                                  ((unsigned long long)tab.piece[1][j] << 16);
                    const unsigned long long hi = (unsigned long long)tab.piece[2][j] +
                                                  ((unsigned long long)tab.piece[3][j] << 16);
                    if (lo) atomicAdd(s.acc[c].lo + k, lo);
                    if (hi) atomicAdd(s.acc[c].hi + k, hi);
                }
            }
        } else if constexpr (NCH < 0) {
            if (base[0] == 0) continue;
            for (int c = 0; c < nch; c++) {
                if (l[c][0] == NONE) continue;
                uint64_t x = base[0];
                for (int j = 0; j < nch; j++)
                    if (j != c) x = sat_mul(x, m[j][0]);
                if (x != 0) acc_add_global(s.acc[c], l[c][0], x);
            }
        }
    }
}

void launch_down(Ctx &c, int grid, const DownSpec &d) {
    switch (d.nch) {
        case 0: k_down<0><<<grid, ST, 0, c.stream>>>(d); break;
        case 1: k_down<1><<<grid, ST, 0, c.stream>>>(d); break;
        case 2: k_down<2><<<grid, ST, 0, c.stream>>>(d); break;
        case 3: k_down<3><<<grid, ST, 0, c.stream>>>(d); break;
        case 4: k_down<4><<<grid, ST, 0, c.stream>>>(d); break;
        default: k_down<-1><<<grid, ST, 0, c.stream>>>(d); break;
    }
    c.launches++;
}

inline KeyCols key_cols(const QRel &q, const std::vector<int> &cols) {
    KeyCols k{};
    k.ncol = (int)cols.size();
    for (int i = 0; i < k.ncol; i++) k.col[i] = q.F->gkey + (int64_t)cols[i] * q.F->G;
    return k;
}

// Whether the parent's link to child ch goes through a dense table over the
// child's single separator column, and that table's range.
bool dense_link(const QRel &t, const QRel &ch, int64_t *range) {
    if (ch.sep_cols.size() != 1 || ch.F->G == 0 || t.F->G == 0) return false;
    const int col = ch.sep_cols[0];
    *range = (int64_t)ch.R->kmax[col] - (int64_t)ch.R->kmin[col] + 1;
    return *range <= DENSE_MAX && *range <= 4 * (ch.F->G + t.F->G) + 4096;
}

}  // namespace

void tri_free(Ctx &c, QueryState &q);
gj_status tri_summarize(QueryState &q, uint64_t *total_out);
void cyc_free(Ctx &c, QueryState &q);
gj_status cyc_summarize(QueryState &q, uint64_t *total_out);

void query_free_summary(Ctx &c, QueryState &q) {
    if (q.cyc) cyc_free(c, q);
    else tri_free(c, q);
    // arrays inside the slab are forgotten, any other one freed; then the
    // slab once
    auto fr = [&](auto *&p) {
        if (q.slab && (const char *)p >= (const char *)q.slab &&
            (const char *)p < (const char *)q.slab + q.slab_bytes)
            p = nullptr;
        else
            dfree(c, p);
    };
    for (auto &t : q.r) {
        fr(t.S_dev);
        fr(t.L_dev);
        fr(t.seg_id);
        fr(t.seg_first);
        for (auto &l : t.link) fr(l);
        t.link.clear();
        fr(t.w);
        fr(t.off);
        fr(t.msg);
        fr(t.down);
        fr(t.mult);
        fr(t.lgid);
        fr(t.loff);
        fr(t.lw);
        fr(t.lseg_first);
    }
    dfree_bytes(c, q.slab);
    q.slab = nullptr;
    q.slab_bytes = 0;
    q.summarized = false;
}

gj_status summarize(QueryState &q, uint64_t *total_out) {
    if (q.tri) return tri_summarize(q, total_out);
    if (q.cyc) return cyc_summarize(q, total_out);
    Ctx &c = q.ctx();
    query_free_summary(c, q);
    cudaError_t e = cudaSuccess;
    // every per-relation array below comes from one slab (a bump arena on
    // the context while this call runs), unless the context already bumps
    // from an arena of its own
    struct ArenaScope {
        Ctx &c;
        bool active = false;
        char *a;
        size_t size, used;
        bool on;
        explicit ArenaScope(Ctx &cc) : c(cc), a(cc.arena), size(cc.arena_size), used(cc.arena_used), on(cc.arena_on) {}
        void set(void *slab, size_t bytes) {
            active = true;
            c.arena = (char *)slab;
            c.arena_size = bytes;
            c.arena_used = 0;
            c.arena_on = true;
        }
        ~ArenaScope() {
            if (!active) return;
            c.arena = a;
            c.arena_size = size;
            c.arena_used = used;
            c.arena_on = on;
        }
    } arena_scope(c);
    if (!c.arena_on) {
        auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
        size_t sb = 0;
        for (const QRel &t : q.r) {
            const size_t G = (size_t)std::max<int64_t>(t.F->G, 1);
            sb += t.children.size() * al(4 * G);                       // links
            sb += 5 * al(8 * G) + al(4 * G) + al(4);                   // w, off, loff, lw, mult; lgid; L_dev
            if (t.parent >= 0)
                sb += 2 * al(8 * G) + al(4 * G) + 2 * al(4 * (G + 1)) + al(4);   // msg, down; seg_id; seg_first, lseg_first; S_dev
        }
        void *slab = nullptr;
        e = dalloc_bytes(c, &slab, sb);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
        q.slab = slab;
        q.slab_bytes = sb;
    }
    // one block of scratch for the whole summary: every relation's lookback
    // state, every dense link table, every child's down accumulators, |Q|
    std::vector<int64_t> st_off(q.k), dense_off(q.k, -1), dense_range(q.k, 0), acc_off(q.k, -1);
    size_t bytes = 64;
    for (int i = 0; i < q.k; i++) {
        st_off[i] = (int64_t)bytes;
        bytes += 16 * (size_t)(ceil_div(std::max<int64_t>(q.r[i].F->G, 1), UP_TILE) + 1);
    }
    const size_t zero_end = bytes;   // lookback state: cleared to 0
    for (int i = 1; i < q.k; i++) {
        const QRel &ch = q.r[i];
        int64_t range = 0;
        if (dense_link(q.r[ch.parent], ch, &range)) {
            dense_off[i] = (int64_t)bytes;
            dense_range[i] = range;
            bytes += ((size_t)range * 4 + 15) & ~(size_t)15;
        }
    }
    const size_t dense_end = bytes;  // dense tables: cleared to 0xFF (NONE)
    for (int i = 1; i < q.k; i++) {
        acc_off[i] = (int64_t)bytes;
        bytes += (size_t)std::max<int64_t>(q.r[i].F->G, 1) * 20;
        bytes = (bytes + 15) & ~(size_t)15;
    }
    char *scratch = nullptr;
    auto acc_of = [&](int i) {
        const int64_t S = std::max<int64_t>(q.r[i].F->G, 1);
        DownAcc a;
        a.lo = (unsigned long long *)(scratch + acc_off[i]);
        a.hi = a.lo + S;
        a.sat = (unsigned int *)(a.hi + S);
        return a;
    };
#define TRY(x)                                                 \
    do {                                                       \
        e = (x);                                               \
        if (e != cudaSuccess) {                                \
            note_cuda_error(e, __FILE__, __LINE__);            \
            goto fail;                                         \
        }                                                      \
    } while (0)
    {
        TRY(dalloc_bytes(c, (void **)&scratch, bytes));
        if (q.slab) arena_scope.set(q.slab, q.slab_bytes);   // the arrays from here on
        TRY(cudaMemsetAsync(scratch, 0, zero_end, c.stream));
        if (dense_end > zero_end) TRY(cudaMemsetAsync(scratch + zero_end, 0xFF, dense_end - zero_end, c.stream));
        if (bytes > dense_end) TRY(cudaMemsetAsync(scratch + dense_end, 0, bytes - dense_end, c.stream));
        uint64_t *total_dev = (uint64_t *)scratch;
        // upward, leaves to root (reverse preorder): links to the children
        // (whose segments exist by now), then the relation's scan
        for (int pi = q.k - 1; pi >= 0; pi--) {
            const int ti = q.pre[pi];
            QRel &t = q.r[ti];
            const int64_t G = t.F->G;
            t.link.assign(t.children.size(), nullptr);
            for (size_t ci = 0; ci < t.children.size(); ci++) {
                const int chi = t.children[ci];
                QRel &ch = q.r[chi];
                TRY(dalloc(c, &t.link[ci], G));
                if (G == 0) continue;
                if (ch.F->G == 0) {
                    k_fill_u32<<<grid_for(c, G), ST, 0, c.stream>>>(t.link[ci], G, NONE); c.launches++;
                } else if (dense_off[chi] >= 0) {
                    k_link_dense<<<grid_for(c, G), ST, 0, c.stream>>>(
                        t.F->gkey + (int64_t)ch.sep_cols_parent[0] * G, G, ch.R->kmin[ch.sep_cols[0]],
                        (uint64_t)dense_range[chi], (const uint32_t *)(scratch + dense_off[chi]), t.link[ci]); c.launches++;
                } else {
                    k_link_search<<<grid_for(c, G), ST, 0, c.stream>>>(
                        key_cols(t, ch.sep_cols_parent), G, key_cols(ch, ch.sep_cols), ch.seg_first,
                        ch.S_dev, t.link[ci]); c.launches++;
                }
                TRY(cudaGetLastError());
            }
            const bool seg = t.parent >= 0;
            TRY(dalloc(c, &t.w, G));
            TRY(dalloc(c, &t.off, G));
            TRY(dalloc(c, &t.lgid, G));        // L <= G live groups
            TRY(dalloc(c, &t.loff, G));
            TRY(dalloc(c, &t.lw, G));
            TRY(dalloc(c, &t.L_dev, 1));
            if (seg) {
                TRY(dalloc(c, &t.msg, G));      // S <= G segments
                TRY(dalloc(c, &t.seg_id, G));
                TRY(dalloc(c, &t.seg_first, G + 1));
                TRY(dalloc(c, &t.lseg_first, G + 1));
                TRY(dalloc(c, &t.S_dev, 1));
            }
            if (G == 0) {
                TRY(cudaMemsetAsync(t.L_dev, 0, 4, c.stream));
                if (seg) {
                    TRY(cudaMemsetAsync(t.S_dev, 0, 4, c.stream));
                    TRY(cudaMemsetAsync(t.seg_first, 0, 4, c.stream));
                    TRY(cudaMemsetAsync(t.lseg_first, 0, 4, c.stream));
                }
                continue;
            }
            UpSpec u{};
            u.G = G;
            u.gstart = t.F->gstart;
            u.nch = (int)t.children.size();
            for (int ci = 0; ci < u.nch; ci++) {
                u.link[ci] = t.link[ci];
                u.msg[ci] = q.r[t.children[ci]].msg;
            }
            u.seg = seg ? 1 : 0;
            if (seg) u.sep = key_cols(t, t.sep_cols);
            u.w = t.w;
            u.off = t.off;
            u.msg_out = t.msg;
            u.seg_id = t.seg_id;
            u.seg_first = t.seg_first;
            u.S_dev = t.S_dev;
            u.lgid = t.lgid;
            u.loff = t.loff;
            u.lw = t.lw;
            u.lseg_first = t.lseg_first;
            u.L_dev = t.L_dev;
            u.total = seg ? nullptr : total_dev;
            if (seg && dense_off[ti] >= 0) {
                u.dense = (uint32_t *)(scratch + dense_off[ti]);
                u.dense_key = t.F->gkey + (int64_t)t.sep_cols[0] * G;
                u.dense_mn = t.R->kmin[t.sep_cols[0]];
            }
            u.status = (ulonglong2 *)(scratch + st_off[ti] + 16);
            u.counter = (uint32_t *)(scratch + st_off[ti]);
            u.err = c.err;
            TRY(launch_up_scan(c, u));
        }
        // downward, root to leaves (preorder): mult, each child's down
        // message, and the relation's own down message finished
        for (int pi = 0; pi < q.k; pi++) {
            const int ti = q.pre[pi];
            QRel &t = q.r[ti];
            const int64_t G = t.F->G;
            TRY(dalloc(c, &t.mult, G));
            if (t.parent >= 0) TRY(dalloc(c, &t.down, G));   // S <= G
            if (G == 0) continue;
            DownSpec d{};
            d.G = G;
            d.gstart = t.F->gstart;
            d.w = t.w;
            d.mult = t.mult;
            if (t.parent >= 0) {
                d.has_down = 1;
                d.self = acc_of(ti);
                d.seg_id = t.seg_id;
                d.seg_first = t.seg_first;
                d.down_out = t.down;
            }
            d.nch = (int)t.children.size();
            for (int ci = 0; ci < d.nch; ci++) {
                d.link[ci] = t.link[ci];
                d.msg[ci] = q.r[t.children[ci]].msg;
                d.acc[ci] = acc_of(t.children[ci]);
                // links in key order when the child joins the parent's
                // leading factor columns: no combining needed
                const std::vector<int> &sp = q.r[t.children[ci]].sep_cols_parent;
                const std::vector<int> &ord = t.F->order;
                const bool in_order = sp.size() <= ord.size() && std::equal(sp.begin(), sp.end(), ord.begin());
                d.agg[ci] = c.down_combine == 2 || (c.down_combine == 0 && !in_order);
            }
            launch_down(c, grid_for(c, G), d);
            TRY(cudaGetLastError());
        }
        // the one synchronisation: |Q| and the device error word
        {
            uint64_t *h = c.pinned;
            h[0] = 0;
            if (q.r[0].F->G) TRY(cudaMemcpyAsync(h, total_dev, 8, cudaMemcpyDeviceToHost, c.stream));
            TRY(cudaMemcpyAsync(h + 1, c.err, 4, cudaMemcpyDeviceToHost, c.stream));
            dfree(c, scratch);
            TRY(cudaStreamSynchronize(c.stream));
            q.total = h[0];
            uint32_t err = (uint32_t)(h[1] & 0xffffffffu);
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
    dfree(c, scratch);
    return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
}

}  // namespace gj
