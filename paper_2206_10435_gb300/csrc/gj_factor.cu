// gj_factor.cu -- factor construction (Section 3.2, quantitative learning).
//
// A relation's potential is its exact frequency table: the distinct key
// tuples with their counts.  Here it is built by sorting the rows by their
// key tuple and cutting the sorted order into groups:
//
//   1. per key column, min and max (one read of every column);
//   2. each column becomes an unsigned field of ceil(log2(max-min+1)) bits,
//      packed into 64-bit words, most significant column first.  When the
//      key and the row id fit one word together, the row id rides in the low
//      bits and a keys-only LSD radix sort orders the key bits (a stable
//      sort of rows taken in row order keeps equal keys in row order);
//      otherwise (word, row id) pairs are sorted, word by word.  The first
//      pass builds the words from the key columns itself;
//   3. one group scan over the sorted words marks the rows whose key differs
//      from the previous row's, numbers these group heads (a single-pass
//      scan with decoupled lookback) and writes the row order, every group's
//      first position and key values, and the payload columns gathered
//      into group order.
//
// Sorted order is also the order the desummariser walks: groups sharing a
// separator value are contiguous (the separator columns lead the order) and
// inside a group rows keep increasing row id.
#include <algorithm>

#include "gj_lookback.cuh"
#include "gj_state.cuh"

namespace gj {
namespace {

constexpr int FT = 256;

struct ColSet {
    int ncol;
    const int32_t *col[MAX_KEYS];
};

__global__ void k_minmax_init(int nk, int32_t *mm) {
    int c = threadIdx.x;
    if (c < nk) { mm[2 * c] = INT32_MAX; mm[2 * c + 1] = INT32_MIN; }
}

__global__ void k_minmax(ColSet cs, int64_t n, int32_t *mm) {
    int c = blockIdx.y;
    const int32_t *col = cs.col[c];
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    const int64_t stride = (int64_t)gridDim.x * FT;
    int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {   // four loads in flight
        const int32_t v0 = __ldg(col + i), v1 = __ldg(col + i + stride);
        const int32_t v2 = __ldg(col + i + 2 * stride), v3 = __ldg(col + i + 3 * stride);
        lo = min(lo, min(min(v0, v1), min(v2, v3)));
        hi = max(hi, max(max(v0, v1), max(v2, v3)));
    }
    for (; i < n; i += stride) {
        const int32_t v = __ldg(col + i);
        lo = min(lo, v);
        hi = max(hi, v);
    }
    for (int d = 16; d; d >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&mm[2 * c], lo);
        atomicMax(&mm[2 * c + 1], hi);
    }
}

struct PackSpec {
    int ncol;
    const int32_t *col[MAX_KEYS];
    int32_t mn[MAX_KEYS];
    int shift[MAX_KEYS];
};

// keys[i] = packed fields of row (rows ? rows[i] : i); vals[i] = that row
__global__ void k_pack(PackSpec ps, const uint32_t *__restrict__ rows, int64_t n,
                       uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT) {
        uint32_t r = rows ? rows[i] : (uint32_t)i;
        uint64_t k = 0;
#pragma unroll
        for (int c = 0; c < MAX_KEYS; c++) {
            if (c < ps.ncol && ps.shift[c] < 64)
                k |= (uint64_t)((uint32_t)ps.col[c][r] - (uint32_t)ps.mn[c]) << ps.shift[c];
        }
        keys[i] = k;
        vals[i] = r;
    }
}

// keys[i] = packed fields of row rows[i]; pos[i] = i (a position in the
// order rows[] lists the rows in)
__global__ void k_pack_pos(PackSpec ps, const uint32_t *__restrict__ rows, int64_t n,
                           uint64_t *__restrict__ keys, uint32_t *__restrict__ pos) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT) {
        const uint32_t r = rows[i];
        uint64_t k = 0;
#pragma unroll
        for (int c = 0; c < MAX_KEYS; c++) {
            if (c < ps.ncol && ps.shift[c] < 64)
                k |= (uint64_t)((uint32_t)ps.col[c][r] - (uint32_t)ps.mn[c]) << ps.shift[c];
        }
        keys[i] = k;
        pos[i] = (uint32_t)i;
    }
}

// the row ids and the low word in the final order: element i came from
// position pos[i] of the order the low word was sorted in
__global__ void k_compose(const uint32_t *__restrict__ pos, const uint32_t *__restrict__ perm0,
                          const uint64_t *__restrict__ lo0, int64_t n, uint32_t *__restrict__ perm,
                          uint64_t *__restrict__ lo) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT) {
        const uint32_t j = pos[i];
        perm[i] = perm0[j];
        lo[i] = lo0[j];
    }
}

// head[i] = i == 0 || key tuple of perm[i] != key tuple of perm[i-1]
__global__ void k_heads_packed(const uint64_t *__restrict__ keys, int64_t n, uint8_t *head) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT)
        head[i] = (i == 0) || keys[i] != keys[i - 1];
}

__global__ void k_heads_gather(ColSet cs, const uint32_t *__restrict__ perm, int64_t n,
                               uint8_t *head) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT) {
        uint8_t h = (i == 0);
        if (!h) {
            uint32_t a = perm[i], b = perm[i - 1];
            for (int c = 0; c < cs.ncol; c++)
                if (cs.col[c][a] != cs.col[c][b]) { h = 1; break; }
        }
        head[i] = h;
    }
}

__global__ void k_group_compact(ColSet cs, const uint32_t *__restrict__ perm,
                                const uint8_t *__restrict__ head, const uint32_t *__restrict__ gid,
                                int64_t n, int64_t G, uint32_t *gstart, int32_t *gkey) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT) {
        if (!head[i]) continue;
        uint32_t g = gid[i];
        gstart[g] = (uint32_t)i;
        uint32_t r = perm[i];
        for (int c = 0; c < cs.ncol; c++) gkey[(int64_t)c * G + g] = cs.col[c][r];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) gstart[G] = (uint32_t)n;
}

// Where each key column sits in the packed words of a sorted key (the low
// word, or the high one of a two-word key): value = ((word >> shift) &
// (2^bits - 1)) + min.  Columns outside the factor's order (projected
// away) are read through perm instead.
struct UnpackSpec {
    int ncol;
    int col[MAX_KEYS];
    int32_t mn[MAX_KEYS];
    int shift[MAX_KEYS];
    int bits[MAX_KEYS];
    int hi[MAX_KEYS];
    int nother;
    int other_col[MAX_KEYS];
    const int32_t *other[MAX_KEYS];
};

// sorted[c*n + i] = col_c[perm[i]]: the key columns in sorted order, one
// random read per column and row (used when the key spans several words)
__global__ void k_gather_cols(ColSet cs, const uint32_t *__restrict__ perm, int64_t n,
                              int32_t *__restrict__ sorted) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT) {
        uint32_t r = perm[i];
        for (int c = 0; c < cs.ncol; c++) sorted[(int64_t)c * n + i] = cs.col[c][r];
    }
}

// the columns a factor groups by (its order; all key columns unless some
// were projected away)
struct ColIdx {
    int n;
    int idx[MAX_KEYS];
};

__global__ void k_heads_sorted(const int32_t *__restrict__ sorted, ColIdx by, int64_t n, uint8_t *head) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT) {
        uint8_t h = (i == 0);
        for (int k = 0; k < by.n && !h; k++) {
            const int64_t c = by.idx[k];
            h = sorted[c * n + i] != sorted[c * n + i - 1];
        }
        head[i] = h;
    }
}

__global__ void k_group_compact_sorted(const int32_t *__restrict__ sorted, int nk,
                                       const uint8_t *__restrict__ head,
                                       const uint32_t *__restrict__ gid, int64_t n, int64_t G,
                                       uint32_t *gstart, int32_t *gkey) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT) {
        if (!head[i]) continue;
        uint32_t g = gid[i];
        gstart[g] = (uint32_t)i;
        for (int c = 0; c < nk; c++) gkey[(int64_t)c * G + g] = sorted[(int64_t)c * n + i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) gstart[G] = (uint32_t)n;
}

template <class T>
__global__ void k_gather(const T *__restrict__ src, const uint32_t *__restrict__ perm, int64_t n,
                         T *__restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT)
        dst[i] = src[perm[i]];
}

inline int grid_for(Ctx &c, int64_t n) {
    int64_t b = ceil_div(n, FT);
    int64_t cap = (int64_t)c.num_sms * 16;
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

inline int bits_of(uint32_t range) { return range == 0 ? 0 : 32 - __builtin_clz(range); }

}  // namespace

cudaError_t relation_minmax(Ctx &c, Relation &R) {
    if (R.have_minmax) return cudaSuccess;
    R.kmin.assign(R.nk, 0);
    R.kmax.assign(R.nk, 0);
    if (R.n > 0) {
        int32_t *mm = nullptr;
        Temps tmp(c);
        GJ_CUDA_TRY(tmp.alloc(&mm, 2 * R.nk));
        ColSet cs{};
        cs.ncol = R.nk;
        for (int i = 0; i < R.nk; i++) cs.col[i] = R.key[i];
        k_minmax_init<<<1, 32, 0, c.stream>>>(R.nk, mm); c.launches++;
        dim3 grid((unsigned)std::max(1, grid_for(c, R.n) / std::max(1, R.nk)), R.nk);
        k_minmax<<<grid, FT, 0, c.stream>>>(cs, R.n, mm); c.launches++;
        GJ_CUDA_TRY(cudaGetLastError());
        // device->host readbacks go through the pinned buffer, then sync
        int32_t *h = (int32_t *)c.pinned;
        GJ_CUDA_TRY(cudaMemcpyAsync(h, mm, sizeof(int32_t) * 2 * R.nk, cudaMemcpyDeviceToHost, c.stream));
        GJ_CUDA_TRY(cudaStreamSynchronize(c.stream));
        for (int i = 0; i < R.nk; i++) { R.kmin[i] = h[2 * i]; R.kmax[i] = h[2 * i + 1]; }
    }
    R.have_minmax = true;
    return cudaSuccess;
}

void factor_free(Ctx &c, Factor &F) {
    dfree(c, F.perm);
    dfree(c, F.gstart);
    dfree(c, F.gkey);
    for (void *&p : F.pay) dfree(c, p);
    F.pay.clear();
}

namespace {

// ------------------------------------------------------------ group scan
// One pass over the sorted words: a row starts a group when its key differs
// from the previous row's; the groups are numbered by a single-pass scan
// with decoupled lookback, and the same pass writes the row order, every
// group's first position and key values, and the payloads in group order.
//   MODE 0  one word per row, the row id in its low row_bits bits
//   MODE 1  one word per row (the key), row order in perm_in
//   MODE 2  two words per row (hi, lo), row order in perm_in
constexpr int GS_THREADS = 256;
constexpr int GS_ITEMS = 16;
constexpr int GS_TILE = GS_THREADS * GS_ITEMS;

struct GroupScanSpec {
    const uint64_t *lo;           // sorted words (the low word of two)
    const uint64_t *hi;           // MODE 2: the high word
    const uint32_t *perm_in;      // MODE 1, 2
    uint32_t *perm_out;           // MODE 0: the row order taken from the words
    int row_bits;
    UnpackSpec u;                 // where each key column sits in the words
    int np;
    const void *pay_in[MAX_PAYLOADS];
    void *pay_out[MAX_PAYLOADS];
    int pw[MAX_PAYLOADS];
    uint32_t *gstart;             // [G+1]
    int32_t *gkey;                // column c of group g at c * gkey_stride + g
    int64_t gkey_stride;
    uint32_t *gcount;             // G
    unsigned long long *status;   // lookback state, one word per tile
    uint32_t *counter;            // tile counter
    uint32_t *err;
    uint32_t spin_limit;          // polls of a bounded wait
    int stall;                    // failure injection: tile 0 never publishes
};

// shared-memory slot of word q (q = 0 is the previous tile's last word): one
// pad word per 16, so that threads reading 16 consecutive words each are
// free of bank conflicts
__device__ __forceinline__ int gs_slot(int q) { return q + (q >> 4); }
constexpr int GS_SLOTS = GS_TILE + 1 + (GS_TILE + 1) / 16 + 1;

template <int MODE>
__global__ void __launch_bounds__(GS_THREADS, 4)
k_group_scan(GroupScanSpec s, int64_t n) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *s_lo = (uint64_t *)smem;
    uint64_t *s_hi = s_lo + GS_SLOTS;          // MODE 2 only
    __shared__ uint32_t s_wsum[GS_THREADS / 32];
    __shared__ uint32_t s_tile, s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(s.counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * GS_TILE;
    if (base >= n) return;
    const int tile_n = (int)min((int64_t)GS_TILE, n - base);
    {
        // the tile's words, 16 loads in flight per thread
        uint64_t a[GS_ITEMS];
#pragma unroll
        for (int i = 0; i < GS_ITEMS; i++) {
            const int64_t idx = base + i * GS_THREADS + tid;
            a[i] = idx < n ? __ldg((const unsigned long long *)s.lo + idx) : 0ull;
        }
#pragma unroll
        for (int i = 0; i < GS_ITEMS; i++) s_lo[gs_slot(i * GS_THREADS + tid + 1)] = a[i];
        if (MODE == 2) {
#pragma unroll
            for (int i = 0; i < GS_ITEMS; i++) {
                const int64_t idx = base + i * GS_THREADS + tid;
                a[i] = idx < n ? __ldg((const unsigned long long *)s.hi + idx) : 0ull;
            }
#pragma unroll
            for (int i = 0; i < GS_ITEMS; i++) s_hi[gs_slot(i * GS_THREADS + tid + 1)] = a[i];
        }
    }
    if (tid == 0) {
        s_lo[0] = base > 0 ? s.lo[base - 1] : 0ull;
        if (MODE == 2) s_hi[0] = base > 0 ? s.hi[base - 1] : 0ull;
    }
    __syncthreads();
    // heads, row e = i * GS_THREADS + tid: one ballot per warp and i; the
    // tile's head counts per (i, warp) in row order, then their exclusive
    // prefix (warp 0, four entries a lane)
    __shared__ uint32_t s_cnt[GS_ITEMS * (GS_THREADS / 32)];
    __shared__ uint32_t s_hb[GS_ITEMS * (GS_THREADS / 32)];   // the ballots
    static_assert(GS_ITEMS * (GS_THREADS / 32) == 128, "four prefix entries per lane of warp 0");
#pragma unroll
    for (int i = 0; i < GS_ITEMS; i++) {
        const int e = i * GS_THREADS + tid;
        bool h = false;
        if (e < tile_n) {
            const uint64_t a = s_lo[gs_slot(e + 1)], b = s_lo[gs_slot(e)];
            if (MODE == 0) h = (a >> s.row_bits) != (b >> s.row_bits);
            else if (MODE == 1) h = a != b;
            else h = a != b || s_hi[gs_slot(e + 1)] != s_hi[gs_slot(e)];
            h = h || base + e == 0;
        }
        const uint32_t hb = __ballot_sync(0xffffffffu, h);
        if (lane == 0) {
            s_cnt[i * (GS_THREADS / 32) + warp] = __popc(hb);
            s_hb[i * (GS_THREADS / 32) + warp] = hb;
        }
    }
    __syncthreads();
    uint32_t agg = 0;
    if (warp == 0) {
        uint32_t v[4], sum = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) { v[j] = s_cnt[lane * 4 + j]; sum += v[j]; }
        uint32_t x = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        agg = __shfl_sync(0xffffffffu, x, 31);
        uint32_t run = x - sum;
#pragma unroll
        for (int j = 0; j < 4; j++) { s_cnt[lane * 4 + j] = run; run += v[j]; }
        if (lane == 0) s_wsum[0] = agg;
    }
    __syncthreads();
    agg = s_wsum[0];
    // the tile's aggregate goes out first; the row order and the payloads do
    // not depend on the group numbering, so they are gathered while the
    // lookback waits on the predecessors
    // (published by the lane that later publishes the prefix: program order
    // keeps the prefix last)
    const bool silent = s.stall && tile == 0;
    if (warp == GS_THREADS / 32 - 1 && lane == 0 && !silent) publish_aggregate<uint32_t>(s.status, tile, agg);
    const uint64_t rmask = s.row_bits ? ((1ull << s.row_bits) - 1) : 0ull;
    // row order and payloads in group order, coalesced; each thread issues
    // its 16 gathers of a payload column together
    uint32_t r[GS_ITEMS];
#pragma unroll
    for (int i = 0; i < GS_ITEMS; i++) {
        const int e = i * GS_THREADS + tid;
        if (MODE == 0) r[i] = (uint32_t)(s_lo[gs_slot(e + 1)] & rmask);
        else r[i] = e < tile_n ? __ldg(s.perm_in + base + e) : 0u;
    }
    if (MODE == 0) {
#pragma unroll
        for (int i = 0; i < GS_ITEMS; i++) {
            const int e = i * GS_THREADS + tid;
            if (e < tile_n) s.perm_out[base + e] = r[i];
        }
    }
    for (int p = 0; p < s.np; p++) {
        if (s.pw[p] == 8) {
            const unsigned long long *src = (const unsigned long long *)s.pay_in[p];
            unsigned long long *dst = (unsigned long long *)s.pay_out[p];
            unsigned long long v[GS_ITEMS];
#pragma unroll
            for (int i = 0; i < GS_ITEMS; i++) v[i] = i * GS_THREADS + tid < tile_n ? __ldg(src + r[i]) : 0ull;
#pragma unroll
            for (int i = 0; i < GS_ITEMS; i++)
                if (i * GS_THREADS + tid < tile_n) dst[base + i * GS_THREADS + tid] = v[i];
        } else {
            const unsigned int *src = (const unsigned int *)s.pay_in[p];
            unsigned int *dst = (unsigned int *)s.pay_out[p];
            unsigned int v[GS_ITEMS];
#pragma unroll
            for (int i = 0; i < GS_ITEMS; i++) v[i] = i * GS_THREADS + tid < tile_n ? __ldg(src + r[i]) : 0u;
#pragma unroll
            for (int i = 0; i < GS_ITEMS; i++)
                if (i * GS_THREADS + tid < tile_n) dst[base + i * GS_THREADS + tid] = v[i];
        }
    }
    if (warp == GS_THREADS / 32 - 1) {
        const uint32_t carry = warp_lookback_published<uint32_t, AddU32>(s.status, tile, agg, lane, s.err,
                                                                          s.spin_limit);
        if (lane == 0) {
            s_carry = carry;
            if (base + GS_TILE >= n) {   // the last tile: the group count
                *s.gcount = carry + agg;
                s.gstart[carry + agg] = (uint32_t)n;
            }
        }
    }
    __syncthreads();
    // group starts and keys, row e = i * GS_THREADS + tid: the heads of one
    // (i, warp) take consecutive group numbers, so the stores of a warp are
    // contiguous where heads are dense
    const uint32_t carry = s_carry;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll 1
    for (int i = 0; i < GS_ITEMS; i++) {
        const uint32_t hb = s_hb[i * (GS_THREADS / 32) + warp];
        if (!((hb >> lane) & 1u)) continue;
        const int e = i * GS_THREADS + tid;
        const int64_t idx = base + e;
        const uint32_t g = carry + s_cnt[i * (GS_THREADS / 32) + warp] + __popc(hb & lt);
        s.gstart[g] = (uint32_t)idx;
        const uint64_t klo = s_lo[gs_slot(e + 1)], khi = MODE == 2 ? s_hi[gs_slot(e + 1)] : 0ull;
        for (int c = 0; c < s.u.ncol; c++) {
            const uint64_t k = s.u.hi[c] ? khi : klo;
            const uint64_t mask = s.u.bits[c] >= 32 ? 0xFFFFFFFFull : ((1ull << s.u.bits[c]) - 1);
            const uint32_t v = (s.u.shift[c] < 64 ? (uint32_t)((k >> s.u.shift[c]) & mask) : 0u) + (uint32_t)s.u.mn[c];
            s.gkey[(int64_t)s.u.col[c] * s.gkey_stride + g] = (int32_t)v;
        }
        if (s.u.nother) {
            const uint32_t r = MODE == 0 ? (uint32_t)(klo & rmask) : s.perm_in[idx];
            for (int c = 0; c < s.u.nother; c++)
                s.gkey[(int64_t)s.u.other_col[c] * s.gkey_stride + g] = s.u.other[c][r];
        }
    }
}

// ------------------------------------------------------------ run sort
// A key that needs more than one word together with the row id: the rows
// are first sorted by the leading columns with the row id under them
// (keys-only), then every run of rows with equal leading columns is sorted
// by the remaining columns and the row id, by one warp in registers: a
// bitonic network over 32 * E elements (element e = k * 32 + lane, padding
// past the run sorts last).  Runs longer than RUN_MAX are not sorted here;
// a flag tells the host to build that factor the two-word way instead.
constexpr int RUN_MAX = 256;

struct RunSortSpec {
    const uint64_t *a;            // lead << row_bits | row, sorted
    int row_bits;
    const uint32_t *run_start;    // [R + 1]
    const uint32_t *R_dev;        // number of runs
    const uint64_t *rest;         // [n] the remaining columns of each row, packed from bit 0
    uint64_t *hi;                 // out: the leading columns' word
    uint64_t *lo;                 // out: the remaining columns' word
    uint32_t *perm;               // out: row ids
    uint32_t *too_long;           // set when a run exceeds RUN_MAX
};

__device__ __forceinline__ bool kr_greater(uint64_t ka, uint32_t ra, uint64_t kb, uint32_t rb) {
    return ka > kb || (ka == kb && ra > rb);
}

template <int E>
__device__ __forceinline__ void warp_bitonic(uint64_t (&key)[E], uint32_t (&row)[E], int lane) {
    constexpr int N = 32 * E;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                // partners in the same lane: exchange in registers
                const int ks = stride >> 5;
#pragma unroll
                for (int k = 0; k < E; k++) {
                    const int kp = k ^ ks;
                    if (kp > k) {
                        const bool up = ((k * 32 + lane) & size) == 0;
                        if (kr_greater(key[k], row[k], key[kp], row[kp]) == up) {
                            const uint64_t tk = key[k]; key[k] = key[kp]; key[kp] = tk;
                            const uint32_t tr = row[k]; row[k] = row[kp]; row[kp] = tr;
                        }
                    }
                }
            } else {
                // partners in another lane: exchange by shuffle; the lane of
                // the lower element keeps the smaller one on an ascending run
#pragma unroll
                for (int k = 0; k < E; k++) {
                    const uint64_t ok = __shfl_xor_sync(0xffffffffu, key[k], stride);
                    const uint32_t orow = __shfl_xor_sync(0xffffffffu, row[k], stride);
                    const bool up = ((k * 32 + lane) & size) == 0;
                    const bool lower = (lane & stride) == 0;
                    const bool gt = kr_greater(key[k], row[k], ok, orow);
                    if ((lower == up) ? gt : !gt) { key[k] = ok; row[k] = orow; }
                }
            }
        }
    }
}

template <int E>
__device__ __forceinline__ void sort_run(const RunSortSpec &s, uint32_t p0, uint32_t m, int lane) {
    const uint64_t rmask = (1ull << s.row_bits) - 1;
    uint64_t key[E];
    uint32_t row[E];
#pragma unroll
    for (int k = 0; k < E; k++) {
        const uint32_t e = k * 32 + lane;
        row[k] = e < m ? (uint32_t)(__ldg((const unsigned long long *)s.a + p0 + e) & rmask) : 0xffffffffu;
    }
#pragma unroll
    for (int k = 0; k < E; k++) key[k] = row[k] != 0xffffffffu ? __ldg((const unsigned long long *)s.rest + row[k]) : ~0ull;
    warp_bitonic<E>(key, row, lane);
    const uint64_t lead = __ldg((const unsigned long long *)s.a + p0) >> s.row_bits;
#pragma unroll
    for (int k = 0; k < E; k++) {
        const uint32_t e = k * 32 + lane;
        if (e < m) {
            s.hi[p0 + e] = lead;
            s.lo[p0 + e] = key[k];
            s.perm[p0 + e] = row[k];
        }
    }
}

// one warp per run, runs taken in turn
__global__ void __launch_bounds__(256) k_sort_runs(RunSortSpec s) {
    const int lane = threadIdx.x & 31;
    const int64_t nruns = *s.R_dev;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nruns; r += warps) {
        const uint32_t p0 = s.run_start[r];
        const uint32_t m = s.run_start[r + 1] - p0;
        if (m <= 32) sort_run<1>(s, p0, m, lane);
        else if (m <= 64) sort_run<2>(s, p0, m, lane);
        else if (m <= 128) sort_run<4>(s, p0, m, lane);
        else if (m <= RUN_MAX) sort_run<8>(s, p0, m, lane);
        else {
            // too long for the registers: flag it (the host builds this
            // factor another way) and leave valid row ids behind, so that the
            // group scan that follows reads only rows of the relation
            if (lane == 0) atomicOr(s.too_long, 1u);
            const uint64_t rmask = (1ull << s.row_bits) - 1;
            for (uint32_t e = lane; e < m; e += 32) {
                const uint64_t w = s.a[p0 + e];
                s.hi[p0 + e] = w >> s.row_bits;
                s.lo[p0 + e] = 0ull;
                s.perm[p0 + e] = (uint32_t)(w & rmask);
            }
        }
    }
}

// the remaining columns of every row packed into one word, in row order
// (sequential reads), so that the run sort gathers one word per row
__global__ void k_pack_rest(PackSrc ps, int64_t n, uint64_t *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT)
        out[i] = pack_word(ps, i);
}

// run heads of the sorted words: the leading columns differ from the
// previous row's
__global__ void k_run_heads(const uint64_t *__restrict__ a, int row_bits, int64_t n, uint8_t *head) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT)
        head[i] = i == 0 || (a[i] >> row_bits) != (a[i - 1] >> row_bits);
}

__global__ void k_run_starts(const uint8_t *__restrict__ head, const uint32_t *__restrict__ excl, int64_t n,
                             const uint32_t *R_dev, uint32_t *run_start) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT)
        if (head[i]) run_start[excl[i]] = (uint32_t)i;
    if (blockIdx.x == 0 && threadIdx.x == 0) run_start[*R_dev] = (uint32_t)n;
}

// One factor build in two stages, so that the builds of several relations
// share their host synchronisations: the key ranges (for the packed field
// widths) before the sort, and the group counts (for the group arrays)
// after it.
struct FactorBuild {
    Relation *R = nullptr;
    Factor *F = nullptr;
    std::vector<int> bits;
    std::vector<std::vector<int>> words;
    // fused path (keys of at most two words): the group scan wrote gstart,
    // the keys at stride n, the payloads and the count
    bool fused = false;
    uint32_t *gstart = nullptr;    // [n+1]
    int32_t *gkey_n = nullptr;     // [nk*n]
    uint32_t *gcount = nullptr;
    // wide keys sorted by their leading columns, then run by run
    bool force_two = false;        // build the two-word way (a run was too long)
    uint32_t *too_long = nullptr;
    // keys of more than two words
    uint8_t *head = nullptr;
    uint32_t *gid = nullptr;
    int32_t *sorted = nullptr;
};

void fb_free(Ctx &c, FactorBuild &b) {
    dfree(c, b.too_long);
    dfree(c, b.gstart);
    dfree(c, b.gkey_n);
    dfree(c, b.gcount);
    dfree(c, b.head);
    dfree(c, b.gid);
    dfree(c, b.sorted);
}

// the key fields of `order` for the group scan: column cols[i] at bit
// shift[i] of word hi[i]
UnpackSpec unpack_spec(const Relation &R, const std::vector<int> &order,
                       const std::vector<std::vector<int>> &words, const std::vector<int> &bits,
                       int row_bits) {
    UnpackSpec u{};
    for (size_t w = 0; w < words.size(); w++) {
        int shift = w == 0 ? row_bits : 0;
        for (int col : words[w]) {   // least significant first, as packed
            u.col[u.ncol] = col;
            u.mn[u.ncol] = R.kmin[col];
            u.shift[u.ncol] = shift;
            u.bits[u.ncol] = bits[col];
            u.hi[u.ncol] = (int)w;
            shift += bits[col];
            u.ncol++;
        }
    }
    for (int col = 0; col < R.nk; col++) {
        if (std::find(order.begin(), order.end(), col) != order.end()) continue;
        u.other_col[u.nother] = col;
        u.other[u.nother] = R.key[col];
        u.nother++;
    }
    return u;
}

PackSrc pack_src(const Relation &R, const std::vector<int> &wcols, const std::vector<int> &bits,
                 int row_bits) {
    PackSrc ps{};
    ps.ncol = (int)wcols.size();
    ps.row_bits = row_bits;
    int shift = row_bits;
    for (int i = 0; i < ps.ncol; i++) {   // wcols[0] is the least significant
        const int col = wcols[i];
        ps.col[i] = R.key[col];
        ps.mn[i] = R.kmin[col];
        ps.shift[i] = shift;
        shift += bits[col];
    }
    return ps;
}

template <int MODE>
cudaError_t launch_group_scan(Ctx &c, GroupScanSpec &gs, int64_t n) {
    const int64_t tiles = ceil_div(n, GS_TILE);
    unsigned long long *state = nullptr;
    Temps tmp(c);
    GJ_CUDA_TRY(tmp.alloc(&state, tiles + 2));
    GJ_CUDA_TRY(cudaMemsetAsync(state, 0, 8 * (tiles + 2), c.stream));
    gs.counter = (uint32_t *)state;
    gs.status = state + 2;
    gs.err = c.err;
    gs.spin_limit = c.spin_limit;
    gs.stall = c.test_stall ? 1 : 0;
    const size_t smem = (size_t)GS_SLOTS * 8 * (MODE == 2 ? 2 : 1);
    GJ_CUDA_TRY(cudaFuncSetAttribute(k_group_scan<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_group_scan<MODE><<<(unsigned)tiles, GS_THREADS, smem, c.stream>>>(gs, n); c.launches++;
    return cudaGetLastError();
}

// The leading columns of `order` that fit one word with the row id, when
// the remaining ones fit another: their number, else 0.
int run_split(const std::vector<int> &order, const std::vector<int> &bits, int row_bits) {
    int nlead = 0, used = row_bits;
    while (nlead < (int)order.size() && used + bits[order[nlead]] <= 64) used += bits[order[nlead++]];
    if (nlead == 0 || nlead == (int)order.size()) return 0;
    int rest = 0;
    for (size_t i = nlead; i < order.size(); i++) rest += bits[order[i]];
    return rest <= 64 ? nlead : 0;
}

// stage 1 (key ranges known): rows sorted by the key tuple; keys of one or
// two words go straight on to the group scan (the group count lands in
// b.gcount), longer keys mark and number their group heads
cudaError_t fb_sort(Ctx &c, FactorBuild &b) {
    Relation &R = *b.R;
    Factor &F = *b.F;
    const std::vector<int> &order = F.order;
    F.n = R.n;
    const int64_t n = R.n;
    if (n == 0) {
        GJ_CUDA_TRY(dalloc(c, &F.perm, 1));
        return cudaSuccess;
    }
    // field widths, least significant column last in `order`
    std::vector<int> &bits = b.bits;
    bits.assign(R.nk, 0);
    for (int i = 0; i < R.nk; i++)
        bits[i] = bits_of((uint32_t)((int64_t)R.kmax[i] - (int64_t)R.kmin[i]));
    int kbits = 0;
    for (int col : order) kbits += bits[col];
    const int row_bits = bits_of((uint32_t)(n - 1));
    // cut the order into words of <= 64 bits, starting from the least
    // significant column
    std::vector<std::vector<int>> &words = b.words;
    {
        std::vector<int> cur;
        int used = 0;
        for (int i = (int)order.size() - 1; i >= 0; i--) {
            int col = order[i];
            if (used + bits[col] > 64 && !cur.empty()) {
                words.push_back(cur);
                cur.clear();
                used = 0;
            }
            cur.push_back(col);
            used += bits[col];
        }
        if (!cur.empty()) words.push_back(cur);
    }
    if (words.size() <= 2) {
        // the fused path: sort, then one group scan
        b.fused = true;
        GroupScanSpec gs{};
        GJ_CUDA_TRY(dalloc(c, &b.gstart, n + 1));
        GJ_CUDA_TRY(dalloc(c, &b.gkey_n, (size_t)R.nk * n));
        GJ_CUDA_TRY(dalloc(c, &b.gcount, 1));
        for (int p = 0; p < R.np; p++) {
            void *d = nullptr;
            GJ_CUDA_TRY(dalloc_bytes(c, &d, (size_t)R.pw[p] * n));
            F.pay.push_back(d);
            gs.pay_in[p] = R.pay[p];
            gs.pay_out[p] = d;
            gs.pw[p] = R.pw[p];
        }
        gs.np = R.np;
        gs.gstart = b.gstart;
        gs.gkey = b.gkey_n;
        gs.gkey_stride = n;
        gs.gcount = b.gcount;
        // temporaries of this build, freed on every way out
        Temps tmp(c);
        uint64_t *k1 = nullptr, *k2 = nullptr, *kres = nullptr;
        GJ_CUDA_TRY(tmp.alloc(&k1, n));
        GJ_CUDA_TRY(tmp.alloc(&k2, n));
        if (words.size() == 1 && kbits + row_bits <= 64) {
            // MODE 0: the row id rides under the key; a keys-only sort of the
            // key bits
            PackSrc ps = pack_src(R, words[0], bits, row_bits);
            GJ_CUDA_TRY(radix_sort_words(c, &ps, k1, k2, nullptr, nullptr, n, row_bits, kbits, &kres, nullptr));
            GJ_CUDA_TRY(dalloc(c, &F.perm, n));
            gs.lo = kres;
            gs.perm_out = F.perm;
            gs.row_bits = row_bits;
            gs.u = unpack_spec(R, order, words, bits, row_bits);
            GJ_CUDA_TRY(launch_group_scan<0>(c, gs, n));
        } else if (words.size() == 1) {
            // MODE 1: (key, row id) pairs
            uint32_t *v1 = nullptr, *v2 = nullptr, *vres = nullptr;
            GJ_CUDA_TRY(tmp.alloc(&v1, n));
            GJ_CUDA_TRY(tmp.alloc(&v2, n));
            PackSrc ps = pack_src(R, words[0], bits, 0);
            GJ_CUDA_TRY(radix_sort_words(c, &ps, k1, k2, v1, v2, n, 0, kbits, &kres, &vres));
            // the sorted row ids become the factor's row order
            F.perm = vres;
            tmp.keep(vres);
            gs.lo = kres;
            gs.perm_in = F.perm;
            gs.u = unpack_spec(R, order, words, bits, 0);
            GJ_CUDA_TRY(launch_group_scan<1>(c, gs, n));
        } else if (int nlead = run_split(order, bits, row_bits); !b.force_two && nlead > 0) {
            // the leading columns with the row id under them (keys-only),
            // then each run of equal leading columns sorted by the rest in
            // registers; the group scan then reads (lead, rest) words
            std::vector<int> lead(order.begin(), order.begin() + nlead);
            std::vector<int> rest(order.begin() + nlead, order.end());
            std::reverse(lead.begin(), lead.end());   // least significant first
            std::reverse(rest.begin(), rest.end());
            int lead_bits = 0;
            for (int col : lead) lead_bits += bits[col];
            PackSrc pa = pack_src(R, lead, bits, row_bits);
            GJ_CUDA_TRY(radix_sort_words(c, &pa, k1, k2, nullptr, nullptr, n, row_bits, lead_bits, &kres, nullptr));
            uint8_t *head = nullptr;
            uint32_t *excl = nullptr, *run_start = nullptr, *R_dev = nullptr;
            GJ_CUDA_TRY(tmp.alloc(&head, n));
            GJ_CUDA_TRY(tmp.alloc(&excl, n));
            GJ_CUDA_TRY(tmp.alloc(&run_start, n + 1));
            GJ_CUDA_TRY(tmp.alloc(&R_dev, 1));
            k_run_heads<<<grid_for(c, n), FT, 0, c.stream>>>(kres, row_bits, n, head); c.launches++;
            GJ_CUDA_TRY(cudaGetLastError());
            GJ_CUDA_TRY(scan_u32(c, nullptr, head, excl, n, R_dev));
            k_run_starts<<<grid_for(c, n), FT, 0, c.stream>>>(head, excl, n, R_dev, run_start); c.launches++;
            GJ_CUDA_TRY(cudaGetLastError());
            uint64_t *hiw = nullptr;
            GJ_CUDA_TRY(tmp.alloc(&hiw, n));
            GJ_CUDA_TRY(dalloc(c, &F.perm, n));
            GJ_CUDA_TRY(dalloc(c, &b.too_long, 1));
            GJ_CUDA_TRY(cudaMemsetAsync(b.too_long, 0, 4, c.stream));
            uint64_t *low = kres == k1 ? k2 : k1;
            RunSortSpec rs{};
            rs.a = kres;
            rs.row_bits = row_bits;
            rs.run_start = run_start;
            rs.R_dev = R_dev;
            uint64_t *restw = nullptr;
            GJ_CUDA_TRY(tmp.alloc(&restw, n));
            k_pack_rest<<<grid_for(c, n), FT, 0, c.stream>>>(pack_src(R, rest, bits, 0), n, restw); c.launches++;
            GJ_CUDA_TRY(cudaGetLastError());
            rs.rest = restw;
            rs.hi = hiw;
            rs.lo = low;
            rs.perm = F.perm;
            rs.too_long = b.too_long;
            k_sort_runs<<<c.num_sms * 8, 256, 0, c.stream>>>(rs); c.launches++;
            GJ_CUDA_TRY(cudaGetLastError());
            tmp.free(head);
            tmp.free(excl);
            tmp.free(run_start);
            tmp.free(R_dev);
            tmp.free(restw);
            gs.lo = low;
            gs.hi = hiw;
            gs.perm_in = F.perm;
            gs.u = unpack_spec(R, order, {rest, lead}, bits, 0);
            GJ_CUDA_TRY(launch_group_scan<2>(c, gs, n));
        } else {
            // MODE 2: the low word sorts with row ids; the high word sorts
            // carrying positions in the low word's order, and one gather then
            // brings the row ids and the low word into the final order
            uint32_t *v1 = nullptr, *v2 = nullptr, *perm0 = nullptr;
            GJ_CUDA_TRY(tmp.alloc(&v1, n));
            GJ_CUDA_TRY(tmp.alloc(&v2, n));
            PackSrc ps = pack_src(R, words[0], bits, 0);
            int lo_bits = 0;
            for (int col : words[0]) lo_bits += bits[col];
            uint64_t *lo_sorted = nullptr;
            GJ_CUDA_TRY(radix_sort_words(c, &ps, k1, k2, v1, v2, n, 0, lo_bits, &lo_sorted, &perm0));
            uint32_t *vfree = perm0 == v1 ? v2 : v1;   // free buffer of n values
            uint64_t *kfree = lo_sorted == k1 ? k2 : k1;
            PackSpec ph{};
            ph.ncol = (int)words[1].size();
            int shift = 0;
            for (int i = 0; i < ph.ncol; i++) {
                const int col = words[1][i];
                ph.col[i] = R.key[col];
                ph.mn[i] = R.kmin[col];
                ph.shift[i] = shift;
                shift += bits[col];
            }
            uint64_t *h1 = nullptr, *hres = nullptr;
            uint32_t *pos2 = nullptr, *pres = nullptr;
            GJ_CUDA_TRY(tmp.alloc(&h1, n));
            GJ_CUDA_TRY(tmp.alloc(&pos2, n));
            k_pack_pos<<<grid_for(c, n), FT, 0, c.stream>>>(ph, perm0, n, kfree, vfree); c.launches++;
            GJ_CUDA_TRY(cudaGetLastError());
            GJ_CUDA_TRY(radix_sort_words(c, nullptr, kfree, h1, vfree, pos2, n, 0, shift, &hres, &pres));
            uint64_t *lo_final = hres == kfree ? h1 : kfree;   // the buffer hres does not hold
            uint32_t *perm = pres == vfree ? pos2 : vfree;
            k_compose<<<grid_for(c, n), FT, 0, c.stream>>>(pres, perm0, lo_sorted, n, perm, lo_final); c.launches++;
            GJ_CUDA_TRY(cudaGetLastError());
            F.perm = perm;
            tmp.keep(perm);
            gs.lo = lo_final;
            gs.hi = hres;
            gs.perm_in = F.perm;
            gs.u = unpack_spec(R, order, words, bits, 0);
            GJ_CUDA_TRY(launch_group_scan<2>(c, gs, n));
        }
        return cudaSuccess;
    }
    // keys of three or more words: (word, row id) sorts word by word, then
    // the key columns are brought into sorted order once and the groups are
    // found with sequential reads
    GJ_CUDA_TRY(dalloc(c, &F.perm, n));
    uint64_t *keys = nullptr;
    Temps tmp(c);
    GJ_CUDA_TRY(tmp.alloc(&keys, n));
    for (size_t w = 0; w < words.size(); w++) {   // least significant word first
        const std::vector<int> &wcols = words[w];
        PackSpec ps{};
        ps.ncol = (int)wcols.size();
        int shift = 0;
        for (int i = 0; i < ps.ncol; i++) {   // wcols[0] is the least significant
            int col = wcols[i];
            ps.col[i] = R.key[col];
            ps.mn[i] = R.kmin[col];
            ps.shift[i] = shift;
            shift += bits[col];
        }
        k_pack<<<grid_for(c, n), FT, 0, c.stream>>>(ps, w == 0 ? nullptr : F.perm, n, keys, F.perm); c.launches++;
        GJ_CUDA_TRY(cudaGetLastError());
        GJ_CUDA_TRY(radix_sort_u64_u32(c, keys, F.perm, n, shift));
    }
    tmp.free(keys);
    GJ_CUDA_TRY(dalloc(c, &b.head, n));
    GJ_CUDA_TRY(dalloc(c, &b.gid, n));
    GJ_CUDA_TRY(dalloc(c, &b.gcount, 1));
    ColSet all{};
    all.ncol = R.nk;
    for (int i = 0; i < R.nk; i++) all.col[i] = R.key[i];
    GJ_CUDA_TRY(dalloc(c, &b.sorted, (size_t)R.nk * n));
    k_gather_cols<<<grid_for(c, n), FT, 0, c.stream>>>(all, F.perm, n, b.sorted); c.launches++;
    ColIdx by{};
    by.n = (int)order.size();
    for (int i = 0; i < by.n; i++) by.idx[i] = order[i];
    k_heads_sorted<<<grid_for(c, n), FT, 0, c.stream>>>(b.sorted, by, n, b.head); c.launches++;
    GJ_CUDA_TRY(cudaGetLastError());
    GJ_CUDA_TRY(scan_u32(c, nullptr, b.head, b.gid, n, b.gcount));
    return cudaSuccess;
}

// stage 2 (group count G known): the group arrays at their final size,
// payloads in group order; frees the stage's temporaries
cudaError_t fb_groups(Ctx &c, FactorBuild &b, int64_t G) {
    Relation &R = *b.R;
    Factor &F = *b.F;
    const int64_t n = R.n;
    if (n == 0) {
        F.G = 0;
        GJ_CUDA_TRY(dalloc(c, &F.gstart, 1));
        GJ_CUDA_TRY(cudaMemsetAsync(F.gstart, 0, sizeof(uint32_t), c.stream));
        GJ_CUDA_TRY(dalloc(c, &F.gkey, 1));
        for (int p = 0; p < R.np; p++) {
            void *d = nullptr;
            GJ_CUDA_TRY(dalloc_bytes(c, &d, 16));
            F.pay.push_back(d);
        }
        return cudaSuccess;
    }
    F.G = G;
    if (b.fused) {
        // group starts stay in their n + 1 slots; the keys move from stride
        // n to stride G
        F.gstart = b.gstart;
        b.gstart = nullptr;
        GJ_CUDA_TRY(dalloc(c, &F.gkey, (size_t)R.nk * G));
        if (G > 0)
            GJ_CUDA_TRY(cudaMemcpy2DAsync(F.gkey, sizeof(int32_t) * G, b.gkey_n, sizeof(int32_t) * n,
                                          sizeof(int32_t) * G, R.nk, cudaMemcpyDeviceToDevice, c.stream));
        fb_free(c, b);
        return cudaSuccess;
    }
    GJ_CUDA_TRY(dalloc(c, &F.gstart, F.G + 1));
    GJ_CUDA_TRY(dalloc(c, &F.gkey, (size_t)R.nk * F.G));
    k_group_compact_sorted<<<grid_for(c, n), FT, 0, c.stream>>>(b.sorted, R.nk, b.head, b.gid, n, F.G,
                                                                F.gstart, F.gkey); c.launches++;
    GJ_CUDA_TRY(cudaGetLastError());
    for (int p = 0; p < R.np; p++) {
        void *d = nullptr;
        GJ_CUDA_TRY(dalloc_bytes(c, &d, (size_t)R.pw[p] * n));
        if (R.pw[p] == 8) {
            k_gather<uint64_t><<<grid_for(c, n), FT, 0, c.stream>>>(
                (const uint64_t *)R.pay[p], F.perm, n, (uint64_t *)d); c.launches++;
        } else {
            k_gather<uint32_t><<<grid_for(c, n), FT, 0, c.stream>>>(
                (const uint32_t *)R.pay[p], F.perm, n, (uint32_t *)d); c.launches++;
        }
        GJ_CUDA_TRY(cudaGetLastError());
        F.pay.push_back(d);
    }
    fb_free(c, b);
    return cudaSuccess;
}

}  // namespace

// Builds the factors F[i] (order set) of relations R[i] together: one
// readback of every missing key range, the sorts, one readback of every
// group count, then the group arrays.  On error the caller frees the
// factors (factor_free); temporaries are freed here.
cudaError_t factor_build_many(Ctx &c, const std::vector<Relation *> &R, const std::vector<Factor *> &F) {
    const size_t m = R.size();
    // key ranges of the relations that lack them, one readback
    std::vector<Relation *> need;
    for (Relation *r : R)
        if (!r->have_minmax && std::find(need.begin(), need.end(), r) == need.end()) need.push_back(r);
    size_t words_mm = 0;
    for (Relation *r : need) words_mm += 2 * r->nk;
    if (words_mm * 4 > (1 << 16) || m * 8 > (1 << 16)) return cudaErrorInvalidValue;
    if (words_mm) {
        int32_t *mm = nullptr;
        Temps tmp(c);
        GJ_CUDA_TRY(tmp.alloc(&mm, words_mm));
        size_t off = 0;
        for (Relation *r : need) {
            if (r->n > 0) {
                ColSet cs{};
                cs.ncol = r->nk;
                for (int i = 0; i < r->nk; i++) cs.col[i] = r->key[i];
                k_minmax_init<<<1, 32, 0, c.stream>>>(r->nk, mm + off); c.launches++;
                dim3 grid((unsigned)std::max(1, grid_for(c, r->n) / std::max(1, r->nk)), r->nk);
                k_minmax<<<grid, FT, 0, c.stream>>>(cs, r->n, mm + off); c.launches++;
                GJ_CUDA_TRY(cudaGetLastError());
            }
            off += 2 * r->nk;
        }
        // device->host readbacks go through the pinned buffer, then sync
        int32_t *h = (int32_t *)c.pinned;
        GJ_CUDA_TRY(cudaMemcpyAsync(h, mm, sizeof(int32_t) * words_mm, cudaMemcpyDeviceToHost, c.stream));
        GJ_CUDA_TRY(cudaStreamSynchronize(c.stream));
        off = 0;
        for (Relation *r : need) {
            r->kmin.assign(r->nk, 0);
            r->kmax.assign(r->nk, 0);
            if (r->n > 0)
                for (int i = 0; i < r->nk; i++) { r->kmin[i] = h[off + 2 * i]; r->kmax[i] = h[off + 2 * i + 1]; }
            r->have_minmax = true;
            off += 2 * r->nk;
        }
    }
    std::vector<FactorBuild> b(m);
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < m && e == cudaSuccess; i++) {
        b[i].R = R[i];
        b[i].F = F[i];
        e = fb_sort(c, b[i]);
    }
    // group counts (and whether a run of a wide key was too long for the
    // run sort), one readback
    uint32_t *hg = (uint32_t *)c.pinned;
    std::vector<int64_t> G(m, 0);
    for (int round = 0; round < 2 && e == cudaSuccess; round++) {
        for (size_t i = 0; i < m; i++) hg[m + i] = 0;
        for (size_t i = 0; i < m && e == cudaSuccess; i++) {
            if (b[i].gcount) e = cudaMemcpyAsync(hg + i, b[i].gcount, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream);
            if (e == cudaSuccess && b[i].too_long)
                e = cudaMemcpyAsync(hg + m + i, b[i].too_long, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        if (e != cudaSuccess) break;
        bool redo = false;
        for (size_t i = 0; i < m; i++) {
            G[i] = b[i].gcount ? (int64_t)hg[i] : 0;
            if (hg[m + i]) {
                // a run longer than the run sort takes: build it the two-word way
                fb_free(c, b[i]);
                factor_free(c, *b[i].F);
                b[i] = FactorBuild{};
                b[i].R = R[i];
                b[i].F = F[i];
                b[i].force_two = true;
                if (e == cudaSuccess) e = fb_sort(c, b[i]);
                redo = true;
            }
        }
        if (!redo) break;
    }
    for (size_t i = 0; i < m && e == cudaSuccess; i++) e = fb_groups(c, b[i], G[i]);
    if (e != cudaSuccess) {
        note_cuda_error(e, __FILE__, __LINE__);
        for (auto &x : b) fb_free(c, x);
    }
    return e;
}

cudaError_t factor_build(Ctx &c, Relation &R, const std::vector<int> &order, Factor &F) {
    F.order = order;
    return factor_build_many(c, {&R}, {&F});
}

}  // namespace gj

namespace gj {

cudaError_t radix_sort_u64_u32_in(Ctx &c, uint64_t *keys, uint32_t *vals, int64_t n, int bits,
                                  uint64_t *k2, uint32_t *v2, uint32_t *hist,
                                  unsigned long long *status, int64_t status_tiles);
cudaError_t scan_u32_in(Ctx &c, const uint32_t *in, const uint8_t *flags, uint32_t *out,
                        int64_t n, uint32_t *total_dev, void *state_mem, size_t state_bytes);

// Factor construction of key columns `cols` (device, n rows) with every
// scratch buffer supplied by the caller (no device allocation).  Writes
// perm[n], gstart[G+1] and gkey[nk*G] (column c of group g at c*G + g) and
// *G_out.  Same steps and kernels as factor_build.
cudaError_t factor_build_in(Ctx &c, const int32_t *const *cols, int nk, int64_t n,
                            const std::vector<int> &order, uint32_t *perm, uint32_t *gstart,
                            int32_t *gkey, int64_t *G_out, const FactorScratch &s) {
    *G_out = 0;
    if (n == 0) return cudaMemsetAsync(gstart, 0, sizeof(uint32_t), c.stream);
    ColSet all{};
    all.ncol = nk;
    for (int i = 0; i < nk; i++) all.col[i] = cols[i];
    // 1. min/max per column, read back through host memory on the stack
    k_minmax_init<<<1, 32, 0, c.stream>>>(nk, s.mm); c.launches++;
    dim3 grid((unsigned)std::max(1, grid_for(c, n) / std::max(1, nk)), nk);
    k_minmax<<<grid, FT, 0, c.stream>>>(all, n, s.mm); c.launches++;
    GJ_CUDA_TRY(cudaGetLastError());
    int32_t mm[2 * MAX_KEYS];
    GJ_CUDA_TRY(cudaMemcpyAsync(mm, s.mm, sizeof(int32_t) * 2 * nk, cudaMemcpyDeviceToHost, c.stream));
    GJ_CUDA_TRY(cudaStreamSynchronize(c.stream));
    std::vector<int> bits(nk);
    for (int i = 0; i < nk; i++) bits[i] = bits_of((uint32_t)((int64_t)mm[2 * i + 1] - (int64_t)mm[2 * i]));
    // 2. packed words, least significant first, each sorted stably
    std::vector<std::vector<int>> words;
    {
        std::vector<int> cur;
        int used = 0;
        for (int i = (int)order.size() - 1; i >= 0; i--) {
            int col = order[i];
            if (used + bits[col] > 64 && !cur.empty()) {
                words.push_back(cur);
                cur.clear();
                used = 0;
            }
            cur.push_back(col);
            used += bits[col];
        }
        if (!cur.empty()) words.push_back(cur);
    }
    bool first = true;
    for (auto &wcols : words) {
        PackSpec ps{};
        ps.ncol = (int)wcols.size();
        int shift = 0;
        for (int i = 0; i < ps.ncol; i++) {
            int col = wcols[i];
            ps.col[i] = cols[col];
            ps.mn[i] = mm[2 * col];
            ps.shift[i] = shift;
            shift += bits[col];
        }
        k_pack<<<grid_for(c, n), FT, 0, c.stream>>>(ps, first ? nullptr : perm, n, s.keys, perm); c.launches++;
        GJ_CUDA_TRY(cudaGetLastError());
        GJ_CUDA_TRY(radix_sort_u64_u32_in(c, s.keys, perm, n, shift, s.k2, s.v2, s.hist, s.status,
                                          s.status_tiles));
        first = false;
    }
    // 3. group heads and ids
    if (words.size() == 1) {
        k_heads_packed<<<grid_for(c, n), FT, 0, c.stream>>>(s.keys, n, s.head); c.launches++;
    } else {
        k_heads_gather<<<grid_for(c, n), FT, 0, c.stream>>>(all, perm, n, s.head); c.launches++;
    }
    GJ_CUDA_TRY(cudaGetLastError());
    GJ_CUDA_TRY(scan_u32_in(c, nullptr, s.head, s.gid, n, s.gcount, s.scan_state, s.scan_state_bytes));
    uint32_t G = 0;
    GJ_CUDA_TRY(cudaMemcpyAsync(&G, s.gcount, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    GJ_CUDA_TRY(cudaStreamSynchronize(c.stream));
    // 4. group starts and key values
    k_group_compact<<<grid_for(c, n), FT, 0, c.stream>>>(all, perm, s.head, s.gid, n, G, gstart,
                                                         gkey); c.launches++;
    GJ_CUDA_TRY(cudaGetLastError());
    *G_out = G;
    return cudaSuccess;
}

}  // namespace gj
