// gj_scan.cu -- single-pass exclusive prefix sums with decoupled lookback.
//
// One launch per scan: every CTA takes the next tile id from a global
// counter (so a tile only ever waits on tiles that are already running);
// for a count held in device memory a grid of resident CTAs keeps taking
// tiles until the elements run out.  For every tile a CTA scans the tile,
// publishes the tile's aggregate, looks back over its
// predecessors' published aggregates/prefixes to find its carry-in, and
// publishes its inclusive prefix.  Polls of a predecessor's flag are bounded
// by SPIN_LIMIT; on expiry the kernel records ERRF_TIMEOUT and carries on,
// so a stuck predecessor can never hang the GPU.
//
// The segmented variant scans pairs (head, value) under
//   (h1, v1) . (h2, v2) = (h1 | h2, h2 ? v2 : v1 + v2),
// which restarts the sum at every segment head; it is used for the offsets
// of key tuples inside their separator segment and for the messages
// (segment sums) of the upward pass.
#include <algorithm>

#include "gj_lookback.cuh"

namespace gj {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr uint32_t F_AGG = 1u, F_PREFIX = 2u, F_HEAD = 4u;   // segmented scans' flags

template <int PAD>
__device__ __forceinline__ int padded(int e) { return e + e / PAD; }

template <class T, class Op, int ITEMS, bool SEG, bool PERSIST>
__global__ void __launch_bounds__(SCAN_THREADS)
k_scan(const T *__restrict__ in, const uint8_t *__restrict__ flags_as_values,
       const uint8_t *__restrict__ heads, T *__restrict__ out, int64_t n,
       uint32_t *tile_counter, uint32_t *st_flag, T *st_agg, T *st_inc, T *total,
       T *seg_total, const uint32_t *__restrict__ seg_id, uint32_t *err,
       const uint32_t *n_dev) {
    constexpr int TILE = SCAN_THREADS * ITEMS;
    // one padding element per 128 bytes: the coalesced phases (a warp on 32
    // consecutive elements) and the per-thread phases (a thread on ITEMS
    // consecutive elements, 64 bytes apart between threads) are then both
    // free of bank conflicts
    constexpr int PAD = 128 / (int)sizeof(T);
    __shared__ T s_val[TILE + TILE / PAD];
    __shared__ uint8_t s_head[SEG ? TILE : 1];
    __shared__ T s_warp_v[SCAN_THREADS / 32];
    __shared__ uint32_t s_warp_h[SCAN_THREADS / 32];
    __shared__ uint32_t s_tile;
    __shared__ T s_carry;
    Op op;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // element count held in device memory (arrays sized for a capacity)
    if (n_dev) n = min(n, (int64_t)*n_dev);
    // one tile per CTA (grid = tiles), or PERSIST: a grid of resident CTAs
    // takes tiles in order from the counter until the elements run out (for
    // counts known only on the device); either way a tile only waits on
    // tiles already taken
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        const int64_t base = (int64_t)tile * TILE;
        if (n == 0) {
            if (tile == 0 && tid == 0 && total) *total = T(0);
            return;
        }
        if (base >= n) return;

        // coalesced load into shared memory
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            int64_t idx = base + i * SCAN_THREADS + tid;
            T v = T(0);
            uint8_t h = 0;
            if (idx < n) {
                v = in ? in[idx] : T(flags_as_values[idx] != 0);
                if (SEG) h = heads[idx] != 0;
            }
            s_val[padded<PAD>(i * SCAN_THREADS + tid)] = v;
            if (SEG) s_head[i * SCAN_THREADS + tid] = h;
        }
        __syncthreads();

        // thread-local scan of ITEMS consecutive elements
        T x[ITEMS];
        uint8_t hx[ITEMS];
        T run = T(0);
        uint32_t any_head = 0;
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            x[i] = s_val[padded<PAD>(tid * ITEMS + i)];
            hx[i] = SEG ? s_head[tid * ITEMS + i] : 0;
            if (SEG && hx[i]) { run = x[i]; any_head = 1; }
            else run = op(run, x[i]);
        }
        // warp inclusive scan of (any_head, run)
        T wv = run;
        uint32_t wh = any_head;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T ov = __shfl_up_sync(0xffffffffu, wv, d);
            uint32_t oh = __shfl_up_sync(0xffffffffu, wh, d);
            if (lane >= d) {
                if (!wh) wv = op(ov, wv);
                wh |= oh;
            }
        }
        if (lane == 31) { s_warp_v[warp] = wv; s_warp_h[warp] = wh; }
        // exclusive within warp
        T ex_v = __shfl_up_sync(0xffffffffu, wv, 1);
        uint32_t ex_h = __shfl_up_sync(0xffffffffu, wh, 1);
        if (lane == 0) { ex_v = T(0); ex_h = 0; }
        __syncthreads();
        // prefix over preceding warps
        T pw_v = T(0);
        uint32_t pw_h = 0;
        for (int w = 0; w < warp; w++) {
            if (s_warp_h[w]) { pw_v = s_warp_v[w]; pw_h = 1; }
            else pw_v = op(pw_v, s_warp_v[w]);
        }
        // combine: thread exclusive = (preceding warps) . (exclusive within warp)
        T th_v = ex_h ? ex_v : op(pw_v, ex_v);
        uint32_t th_h = ex_h | pw_h;

        // tile aggregate and lookback
        if constexpr (!SEG) {
            if (warp == SCAN_THREADS / 32 - 1) {
                const T agg_v = __shfl_sync(0xffffffffu, op(pw_v, wv), 31);
                const T carry = warp_lookback<T, Op>(
                    reinterpret_cast<typename TileStatus<T>::W *>(st_agg), tile, agg_v, lane, err);
                if (lane == 31) {
                    s_carry = carry;
                    if (total && base + TILE >= n) *total = op(carry, agg_v);
                }
            }
        } else if (tid == SCAN_THREADS - 1) {
            T agg_v = wh ? wv : op(pw_v, wv);
            uint32_t agg_h = wh | pw_h;
            T carry = T(0);
            if (tile == 0) {
                st_inc[tile] = agg_v;
                __threadfence();
                atomicExch(&st_flag[tile], F_PREFIX | (agg_h ? F_HEAD : 0u));
            } else {
                // the aggregate and the inclusive prefix live in separate slots,
                // so a reader that saw F_AGG never reads the later prefix
                st_agg[tile] = agg_v;
                __threadfence();
                atomicExch(&st_flag[tile], F_AGG | (agg_h ? F_HEAD : 0u));
                int64_t p = (int64_t)tile - 1;
                while (p >= 0) {
                    uint32_t f;
                    uint32_t spins = 0;
                    while ((f = ld_volatile(&st_flag[p])) == 0u) {
                        if (++spins > SPIN_LIMIT) { raise_err(err, ERRF_TIMEOUT); f = F_PREFIX; break; }
                    }
                    __threadfence();
                    T v = (f & F_PREFIX) ? ld_volatile(&st_inc[p]) : ld_volatile(&st_agg[p]);
                    carry = op(v, carry);
                    if ((f & F_PREFIX) || (f & F_HEAD)) break;
                    p--;
                }
                T inc = agg_h ? agg_v : op(carry, agg_v);
                st_inc[tile] = inc;
                __threadfence();
                atomicExch(&st_flag[tile], F_PREFIX | (agg_h ? F_HEAD : 0u));
            }
            s_carry = carry;
            if (total && base + TILE >= n) *total = agg_h ? agg_v : op(carry, agg_v);
        }
        __syncthreads();
        T r = th_h ? th_v : op(s_carry, th_v);
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            if (SEG && hx[i]) r = T(0);
            s_val[padded<PAD>(tid * ITEMS + i)] = r;
            r = op(r, x[i]);
            if (SEG && seg_total) {
                int64_t idx = base + tid * ITEMS + i;
                if (idx < n) {
                    bool last = (idx == n - 1) || heads[idx + 1] != 0;
                    if (last) seg_total[seg_id[idx]] = r;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            int64_t idx = base + i * SCAN_THREADS + tid;
            if (idx < n) out[idx] = s_val[padded<PAD>(i * SCAN_THREADS + tid)];
        }
        if (!PERSIST) return;
        __syncthreads();
    }
}

// resident CTAs for a persistent scan grid
inline int64_t scan_grid(Ctx &c, int64_t tiles) {
    return std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)c.num_sms * 8));
}

template <class T, class Op, int ITEMS, bool SEG>
cudaError_t launch_scan(Ctx &c, const T *in, const uint8_t *fv, const uint8_t *heads, T *out,
                        int64_t n, T *total, T *seg_total, const uint32_t *seg_id,
                        const uint32_t *n_dev = nullptr) {
    constexpr int TILE = SCAN_THREADS * ITEMS;
    if (n <= 0) {
        if (total) GJ_CUDA_TRY(cudaMemsetAsync(total, 0, sizeof(T), c.stream));
        return cudaSuccess;
    }
    int64_t tiles = ceil_div(n, TILE);
    if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
    uint32_t *state = nullptr;
    // layout: [counter][pad][flags (tiles)][values (tiles, 8-aligned)]
    size_t flag_bytes = ((size_t)tiles * 4 + 15) & ~(size_t)15;
    size_t bytes = 16 + flag_bytes + 2 * (size_t)tiles * sizeof(T);
    Temps tmp(c);
    GJ_CUDA_TRY(tmp.alloc_bytes((void **)&state, bytes));
    // unsegmented scans keep their status words in the value area: clear it too
    GJ_CUDA_TRY(cudaMemsetAsync(state, 0, !SEG ? bytes : 16 + flag_bytes, c.stream));
    uint32_t *counter = state;
    uint32_t *flags = state + 4;
    T *agg = (T *)((char *)state + 16 + flag_bytes);
    T *inc = agg + tiles;
    if (n_dev)
        k_scan<T, Op, ITEMS, SEG, true><<<(unsigned)scan_grid(c, tiles), SCAN_THREADS, 0, c.stream>>>(
            in, fv, heads, out, n, counter, flags, agg, inc, total, seg_total, seg_id, c.err, n_dev);
    else
        k_scan<T, Op, ITEMS, SEG, false><<<(unsigned)tiles, SCAN_THREADS, 0, c.stream>>>(
            in, fv, heads, out, n, counter, flags, agg, inc, total, seg_total, seg_id, c.err, n_dev);
    c.launches++;
    return cudaGetLastError();
}

}  // namespace

cudaError_t scan_u32(Ctx &c, const uint32_t *in, const uint8_t *flags, uint32_t *out,
                     int64_t n, uint32_t *total_dev) {
    return launch_scan<uint32_t, AddU32, 16, false>(c, in, flags, nullptr, out, n, total_dev,
                                                    nullptr, nullptr);
}

cudaError_t scan_u64_sat(Ctx &c, const uint64_t *in, const uint8_t *heads, uint64_t *out,
                         int64_t n, uint64_t *total_dev, uint64_t *seg_total,
                         const uint32_t *seg_id) {
    if (heads)
        return launch_scan<uint64_t, SatAddU64, 8, true>(c, in, nullptr, heads, out, n,
                                                         total_dev, seg_total, seg_id);
    return launch_scan<uint64_t, SatAddU64, 8, false>(c, in, nullptr, nullptr, out, n,
                                                      total_dev, nullptr, nullptr);
}

cudaError_t scan_u32_dev(Ctx &c, const uint32_t *in, const uint8_t *flags, uint32_t *out,
                         int64_t cap, const uint32_t *n_dev, uint32_t *total_dev) {
    if (cap <= 0) {
        if (total_dev) GJ_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), c.stream));
        return cudaSuccess;
    }
    return launch_scan<uint32_t, AddU32, 16, false>(c, in, flags, nullptr, out, cap, total_dev,
                                                    nullptr, nullptr, n_dev);
}

}  // namespace gj

namespace gj {

// scan_u32 with the lookback state in caller memory (no device allocation):
// state must hold scan_u32_state_bytes(n) bytes.
static_assert(SCAN_THREADS * 16 == SCAN_U32_TILE, "the 32-bit scan tile is exported through gj_internal.cuh");

size_t scan_u32_state_bytes(int64_t n) { return scan_u32_state_bytes_for(n); }

cudaError_t scan_u32_in(Ctx &c, const uint32_t *in, const uint8_t *flags, uint32_t *out,
                        int64_t n, uint32_t *total_dev, void *state_mem, size_t state_bytes) {
    constexpr int TILE = SCAN_THREADS * 16;
    if (n <= 0) {
        if (total_dev) GJ_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), c.stream));
        return cudaSuccess;
    }
    if (state_bytes < scan_u32_state_bytes(n)) return cudaErrorInvalidValue;
    int64_t tiles = ceil_div(n, TILE);
    size_t flag_bytes = ((size_t)tiles * 4 + 15) & ~(size_t)15;
    uint32_t *state = (uint32_t *)state_mem;
    // the status words live in the value area (see k_scan): clear it too
    GJ_CUDA_TRY(cudaMemsetAsync(state, 0, 16 + flag_bytes + 8 * (size_t)tiles, c.stream));
    uint32_t *counter = state;
    uint32_t *fl = state + 4;
    uint32_t *agg = (uint32_t *)((char *)state + 16 + flag_bytes);
    uint32_t *inc = agg + tiles;
    k_scan<uint32_t, AddU32, 16, false, false><<<(unsigned)tiles, SCAN_THREADS, 0, c.stream>>>(
        in, flags, nullptr, out, n, counter, fl, agg, inc, total_dev, nullptr, nullptr, c.err,
        nullptr); c.launches++;
    return cudaGetLastError();
}

}  // namespace gj
