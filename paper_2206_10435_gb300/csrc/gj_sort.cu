// gj_sort.cu -- stable LSD radix sort of (uint64 key, uint32 value) pairs.
//
// Used by factor construction to order a relation's rows by their packed
// join-key tuple (Section 3.2: the frequency table is the run-length form of
// the sorted rows).  8-bit digits, one "onesweep" launch per digit:
//
//   * one upfront pass reads every key once and builds the 256-bin
//     histogram of every digit in shared memory (warp-private bins, then
//     global atomics); a tiny kernel turns them into bucket bases;
//   * per digit, each CTA takes the next tile id from a global counter,
//     ranks its 4096 keys with a warp-level multi-split (peers found by
//     one ballot per digit bit, per-warp bins, no atomics), publishes its per-digit counts,
//     finds each digit's global offset by decoupled lookback over the
//     preceding tiles (bounded polls, ERRF_TIMEOUT on expiry), stages the
//     tile in shared memory in digit order and scatters it so that
//     consecutive threads write consecutive addresses of a bucket.
//
// Stable: ranks follow (tile, warp, item, lane) order, which is input order.
#include <algorithm>

#include "gj_internal.cuh"

namespace gj {
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;       // 4096 keys
constexpr int RS_RADIX = 256;
constexpr int RS_MAX_PASSES = 8;
static_assert(RS_TILE == RADIX_SORT_TILE && RS_RADIX == RADIX_SORT_BINS &&
                  RS_MAX_PASSES == RADIX_SORT_MAX_PASSES,
              "the sort's tile layout is exported through gj_internal.cuh");
constexpr uint64_t ST_AGG = 1ull << 62, ST_PREFIX = 2ull << 62, ST_MASK = (1ull << 62) - 1;
// predecessors whose status a tile reads per round of its lookback
#ifndef RS_LOOKBACK
#define RS_LOOKBACK 4
#endif
// resident CTAs per SM the keys-only kernel is compiled for
#ifndef RS_KEYS_CTAS
#define RS_KEYS_CTAS 4
#endif

template <bool PACK>
__global__ void __launch_bounds__(RS_THREADS)
k_digit_hist(const uint64_t *__restrict__ keys, PackSrc ps, int64_t n, int lo_bit, int passes,
             uint32_t *hist) {
    __shared__ uint32_t sh[RS_MAX_PASSES][RS_RADIX];
    for (int i = threadIdx.x; i < RS_MAX_PASSES * RS_RADIX; i += RS_THREADS) (&sh[0][0])[i] = 0;
    __syncthreads();
    // four words per thread and round, their loads issued together
    const int64_t stride = (int64_t)gridDim.x * RS_THREADS;
    for (int64_t i0 = (int64_t)blockIdx.x * RS_THREADS + threadIdx.x; i0 < n; i0 += 4 * stride) {
        uint64_t k[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t i = i0 + u * stride;
            k[u] = i < n ? (PACK ? pack_word(ps, i) : __ldg((const unsigned long long *)keys + i)) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (i0 + u * stride < n)
                for (int p = 0; p < passes; p++) atomicAdd(&sh[p][(k[u] >> (lo_bit + 8 * p)) & 0xff], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RS_RADIX; i += RS_THREADS) {
        uint32_t v = (&sh[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// hist[p][d] -> exclusive bucket base per pass (one CTA per pass)
__global__ void __launch_bounds__(RS_RADIX) k_hist_to_base(uint32_t *hist) {
    __shared__ uint32_t s[RS_RADIX];
    uint32_t *h = hist + blockIdx.x * RS_RADIX;
    int d = threadIdx.x;
    s[d] = h[d];
    __syncthreads();
    for (int off = 1; off < RS_RADIX; off <<= 1) {
        uint32_t v = d >= off ? s[d - off] : 0u;
        __syncthreads();
        s[d] += v;
        __syncthreads();
    }
    h[d] = s[d] - h[d];
}

__device__ __forceinline__ unsigned long long ld_status(const unsigned long long *q) {
    return *(const volatile unsigned long long *)q;
}

// keys[i] = pack(i), vals[i] = i: a packed sort with nothing to order
__global__ void k_pack_words(PackSrc ps, int64_t n, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    for (int64_t i = (int64_t)blockIdx.x * RS_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * RS_THREADS) {
        keys[i] = pack_word(ps, i);
        if (vals) vals[i] = (uint32_t)i;
    }
}

template <bool VALS, bool PACK>
__global__ void __launch_bounds__(RS_THREADS, VALS ? 3 : RS_KEYS_CTAS)
k_onesweep_t(const uint64_t *__restrict__ kin, PackSrc ps, const uint32_t *__restrict__ vin,
             uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
             const uint32_t *__restrict__ bucket_base, uint32_t *tile_counter,
             unsigned long long *status, uint32_t *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *s_keys = (uint64_t *)smem;                              // RS_TILE
    uint32_t *s_vals = (uint32_t *)(s_keys + RS_TILE);                // RS_TILE (VALS only)
    uint32_t *s_whist = s_vals + (VALS ? RS_TILE : 0);                // RS_WARPS*RS_RADIX
    uint32_t *s_tile_off = s_whist + RS_WARPS * RS_RADIX;             // RS_RADIX
    uint32_t *s_glob = s_tile_off + RS_RADIX;                         // RS_RADIX
    uint32_t *s_misc = s_glob + RS_RADIX;                             // 8

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_misc[0] = atomicAdd(tile_counter, 1u);
    for (int i = tid; i < RS_WARPS * RS_RADIX; i += RS_THREADS) s_whist[i] = 0;
    __syncthreads();
    const uint32_t tile = s_misc[0];
    const int64_t base = (int64_t)tile * RS_TILE;

    uint64_t k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    uint32_t rank[RS_ITEMS];
    const int64_t wbase = base + warp * (RS_ITEMS * 32);
    if (PACK) {
        // pass 0 of a packed sort builds the tile's words from the key
        // columns, staged in shared memory (the value is then the row id, the
        // input position); per column, the thread's 16 loads are issued
        // together
        uint64_t acc[RS_ITEMS];
#pragma unroll
        for (int i = 0; i < RS_ITEMS; i++) {
            const int64_t idx = base + i * RS_THREADS + tid;
            acc[i] = (ps.row_bits && idx < n) ? (uint64_t)idx : 0ull;
        }
        for (int c = 0; c < ps.ncol; c++) {
            if (ps.shift[c] >= 64) continue;
            const int32_t *col = ps.col[c];
            const uint32_t mn = (uint32_t)ps.mn[c];
            const int sh = ps.shift[c];
            uint32_t x[RS_ITEMS];
#pragma unroll
            for (int i = 0; i < RS_ITEMS; i++) {
                const int64_t idx = base + i * RS_THREADS + tid;
                x[i] = idx < n ? (uint32_t)__ldg(col + idx) : mn;
            }
#pragma unroll
            for (int i = 0; i < RS_ITEMS; i++) acc[i] |= (uint64_t)(x[i] - mn) << sh;
        }
#pragma unroll
        for (int i = 0; i < RS_ITEMS; i++) s_keys[i * RS_THREADS + tid] = acc[i];
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t idx = wbase + i * 32 + lane;
        if (idx < n) {
            k[i] = PACK ? s_keys[idx - base] : kin[idx];
            v[i] = VALS ? (PACK ? (uint32_t)idx : vin[idx]) : 0u;
        } else { k[i] = 0; v[i] = 0; }
    }
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t *wh = s_whist + warp * RS_RADIX;
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t idx = wbase + i * 32 + lane;
        bool valid = idx < n;
        uint32_t d = valid ? (uint32_t)((k[i] >> shift) & 0xff) : 0x100u;
        // lanes with the same digit (and validity): one ballot per bit
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < 9; b++) {
            const uint32_t bit = (d >> b) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bal : ~bal;
        }
        int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (valid && lane == leader) {
            old = wh[d];
            wh[d] = old + __popc(peers);
        }
        old = __shfl_sync(0xffffffffu, old, leader);
        rank[i] = old + __popc(peers & lt_mask);
        __syncwarp();
    }
    __syncthreads();

    // per digit: tile count, and per-warp exclusive offsets
    const int d = tid;   // RS_THREADS == RS_RADIX
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; w++) {
        uint32_t c = s_whist[w * RS_RADIX + d];
        s_whist[w * RS_RADIX + d] = cnt;
        cnt += c;
    }
    // publish the tile's count of digit d, then look back for its prefix
    unsigned long long *st = status + (size_t)tile * RS_RADIX;
    atomicExch(&st[d], (unsigned long long)((tile == 0 ? ST_PREFIX : ST_AGG) | cnt));
    // look back RS_LOOKBACK predecessors per round (their
    // status words are read together, then folded nearest first; one that
    // has published nothing yet is polled, bounded, before the fold goes on)
    if (tile == 0) {
        s_glob[d] = bucket_base[d];
    } else {
        uint64_t excl = 0;
        int64_t p = (int64_t)tile - 1;
        bool done = false;
        while (!done && p >= 0) {
            unsigned long long sv[RS_LOOKBACK];
#pragma unroll
            for (int j = 0; j < RS_LOOKBACK; j++)
                sv[j] = p - j >= 0 ? ld_status(status + (size_t)(p - j) * RS_RADIX + d)
                                   : (unsigned long long)ST_PREFIX;
#pragma unroll
            for (int j = 0; j < RS_LOOKBACK; j++) {
                if (!done) {
                    unsigned long long s = sv[j];
                    uint32_t spins = 0;
                    while ((s >> 62) == 0) {
                        if (++spins > SPIN_LIMIT) { raise_err(err, ERRF_TIMEOUT); s = ST_PREFIX; break; }
                        s = ld_status(status + (size_t)(p - j) * RS_RADIX + d);
                    }
                    excl += s & ST_MASK;
                    done = (s & ST_PREFIX) != 0;
                }
            }
            p -= RS_LOOKBACK;
        }
        atomicExch(&st[d], (unsigned long long)(ST_PREFIX | (excl + cnt)));
        s_glob[d] = bucket_base[d] + (uint32_t)excl;
    }
    // tile-local exclusive offsets over digits: a shuffle scan per warp of
    // 32 digits, then the totals of the preceding warps (s_misc holds them;
    // the tile id it held is in a register by now)
    {
        uint32_t x = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) s_misc[warp] = x;
        __syncthreads();
        uint32_t pre = 0;
        for (int w = 0; w < warp; w++) pre += s_misc[w];
        s_tile_off[d] = pre + x - cnt;
    }
    __syncthreads();
    // stage in digit order
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t idx = wbase + i * 32 + lane;
        if (idx < n) {
            uint32_t dg = (uint32_t)((k[i] >> shift) & 0xff);
            uint32_t pos = s_tile_off[dg] + s_whist[warp * RS_RADIX + dg] + rank[i];
            s_keys[pos] = k[i];
            if (VALS) s_vals[pos] = v[i];
        }
    }
    __syncthreads();
    const int64_t tile_n = (n - base) < RS_TILE ? (n - base) : RS_TILE;
#pragma unroll 4
    for (int i = 0; i < RS_ITEMS; i++) {
        int p = i * RS_THREADS + tid;
        if (p < tile_n) {
            uint64_t key = s_keys[p];
            uint32_t dg = (uint32_t)((key >> shift) & 0xff);
            uint32_t dest = s_glob[dg] + (uint32_t)(p - s_tile_off[dg]);
            kout[dest] = key;
            if (VALS) vout[dest] = s_vals[p];
        }
    }
}

// the (key, value) form used by factor construction
constexpr auto k_onesweep = k_onesweep_t<true, false>;

constexpr size_t RS_SMEM = (size_t)RS_TILE * 8 + (size_t)RS_TILE * 4 +
                           (size_t)RS_WARPS * RS_RADIX * 4 + 2 * RS_RADIX * 4 + 8 * 4;
// keys only: no staged values (5 CTAs fit an SM's shared memory)
constexpr size_t RS_SMEM_K = (size_t)RS_TILE * 8 + (size_t)RS_WARPS * RS_RADIX * 4 + 2 * RS_RADIX * 4 + 8 * 4;

}  // namespace

cudaError_t radix_sort_u64_u32(Ctx &c, uint64_t *keys, uint32_t *vals, int64_t n, int bits) {
    if (n <= 1 || bits <= 0) return cudaSuccess;
    if (n > 0x7fffffffLL || bits > 64) return cudaErrorInvalidValue;
    // the limit belongs to the current device: set it on every call (cheap,
    // and right for every device and thread)
    GJ_CUDA_TRY(cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)RS_SMEM));
    const int passes = (bits + 7) / 8;
    const int64_t tiles = ceil_div(n, RS_TILE);
    uint64_t *k2 = nullptr;
    uint32_t *v2 = nullptr, *hist = nullptr, *counters = nullptr;
    unsigned long long *status = nullptr;
    Temps tmp(c);
    GJ_CUDA_TRY(tmp.alloc(&k2, n));
    GJ_CUDA_TRY(tmp.alloc(&v2, n));
    GJ_CUDA_TRY(tmp.alloc(&hist, RS_MAX_PASSES * RS_RADIX + passes));
    GJ_CUDA_TRY(tmp.alloc(&status, (size_t)tiles * RS_RADIX));
    counters = hist + RS_MAX_PASSES * RS_RADIX;
    GJ_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (RS_MAX_PASSES * RS_RADIX + passes),
                                c.stream));
    int hist_blocks = (int)std::min<int64_t>(ceil_div(n, RS_THREADS * 16), (int64_t)c.num_sms * 4);
    if (hist_blocks < 1) hist_blocks = 1;
    k_digit_hist<false><<<hist_blocks, RS_THREADS, 0, c.stream>>>(keys, PackSrc{}, n, 0, passes, hist); c.launches++;
    k_hist_to_base<<<passes, RS_RADIX, 0, c.stream>>>(hist); c.launches++;
    uint64_t *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    for (int p = 0; p < passes; p++) {
        GJ_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(unsigned long long) * tiles * RS_RADIX,
                                    c.stream));
        k_onesweep<<<(unsigned)tiles, RS_THREADS, RS_SMEM, c.stream>>>(
            ka, PackSrc{}, va, kb, vb, n, 8 * p, hist + p * RS_RADIX, counters + p, status, c.err); c.launches++;
        GJ_CUDA_TRY(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        GJ_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, c.stream));
        GJ_CUDA_TRY(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, c.stream));
    }
    return cudaSuccess;
}

}  // namespace gj

namespace gj {

// Same sort with every scratch buffer supplied by the caller (no device
// allocation): k2/v2 hold n entries, hist 8*256 + 8 words, status
// status_tiles*256 words (status_tiles >= ceil(n / 4096)).
cudaError_t radix_sort_u64_u32_in(Ctx &c, uint64_t *keys, uint32_t *vals, int64_t n, int bits,
                                  uint64_t *k2, uint32_t *v2, uint32_t *hist,
                                  unsigned long long *status, int64_t status_tiles) {
    if (n <= 1 || bits <= 0) return cudaSuccess;
    if (n > 0x7fffffffLL || bits > 64) return cudaErrorInvalidValue;
    const int passes = (bits + 7) / 8;
    const int64_t tiles = ceil_div(n, RS_TILE);
    if (tiles > status_tiles) return cudaErrorInvalidValue;
    GJ_CUDA_TRY(cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)RS_SMEM));
    uint32_t *counters = hist + RS_MAX_PASSES * RS_RADIX;
    GJ_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (RS_MAX_PASSES * RS_RADIX + passes),
                                c.stream));
    int hist_blocks = (int)std::min<int64_t>(ceil_div(n, RS_THREADS * 16), (int64_t)c.num_sms * 4);
    if (hist_blocks < 1) hist_blocks = 1;
    k_digit_hist<false><<<hist_blocks, RS_THREADS, 0, c.stream>>>(keys, PackSrc{}, n, 0, passes, hist); c.launches++;
    k_hist_to_base<<<passes, RS_RADIX, 0, c.stream>>>(hist); c.launches++;
    uint64_t *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    for (int p = 0; p < passes; p++) {
        GJ_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(unsigned long long) * tiles * RS_RADIX,
                                    c.stream));
        k_onesweep<<<(unsigned)tiles, RS_THREADS, RS_SMEM, c.stream>>>(
            ka, PackSrc{}, va, kb, vb, n, 8 * p, hist + p * RS_RADIX, counters + p, status, c.err); c.launches++;
        GJ_CUDA_TRY(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        GJ_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, c.stream));
        GJ_CUDA_TRY(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, c.stream));
    }
    return cudaSuccess;
}

}  // namespace gj

namespace gj {

// Sets the keys-only sort kernel's shared-memory limit; call once before
// any capture of radix_sort_keys_u64_in.
cudaError_t radix_sort_keys_prepare() {
    return cudaFuncSetAttribute(k_onesweep_t<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)RS_SMEM);
}

// Keys-only sort with caller scratch (no allocation, capturable in a CUDA
// graph): k2 holds n keys, hist 8*256 + 8 words, status status_tiles*256
// words.  Accepts up to 2^32 - 1 keys.
cudaError_t radix_sort_keys_u64_in(Ctx &c, uint64_t *keys, int64_t n, int bits, uint64_t *k2,
                                   uint32_t *hist, unsigned long long *status,
                                   int64_t status_tiles) {
    if (n <= 1 || bits <= 0) return cudaSuccess;
    if (n > 0xffffffffLL || bits > 64) return cudaErrorInvalidValue;
    const int passes = (bits + 7) / 8;
    const int64_t tiles = ceil_div(n, RS_TILE);
    if (tiles > status_tiles) return cudaErrorInvalidValue;
    uint32_t *counters = hist + RS_MAX_PASSES * RS_RADIX;
    GJ_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (RS_MAX_PASSES * RS_RADIX + passes),
                                c.stream));
    int hist_blocks = (int)std::min<int64_t>(ceil_div(n, RS_THREADS * 16), (int64_t)c.num_sms * 4);
    if (hist_blocks < 1) hist_blocks = 1;
    k_digit_hist<false><<<hist_blocks, RS_THREADS, 0, c.stream>>>(keys, PackSrc{}, n, 0, passes, hist); c.launches++;
    k_hist_to_base<<<passes, RS_RADIX, 0, c.stream>>>(hist); c.launches++;
    uint64_t *ka = keys, *kb = k2;
    for (int p = 0; p < passes; p++) {
        GJ_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(unsigned long long) * tiles * RS_RADIX,
                                    c.stream));
        k_onesweep_t<false, false><<<(unsigned)tiles, RS_THREADS, RS_SMEM, c.stream>>>(
            ka, PackSrc{}, nullptr, kb, nullptr, n, 8 * p, hist + p * RS_RADIX, counters + p, status, c.err); c.launches++;
        GJ_CUDA_TRY(cudaGetLastError());
        std::swap(ka, kb);
    }
    if (ka != keys)
        GJ_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, c.stream));
    return cudaSuccess;
}

}  // namespace gj

namespace gj {

cudaError_t radix_sort_words(Ctx &c, const PackSrc *pack, uint64_t *keys, uint64_t *alt,
                             uint32_t *vals, uint32_t *valt, int64_t n, int lo_bit, int bits,
                             uint64_t **kres, uint32_t **vres) {
    *kres = keys;
    if (vres) *vres = vals;
    if (n > 0x7fffffffLL || bits < 0 || lo_bit < 0 || lo_bit + bits > 64) return cudaErrorInvalidValue;
    const bool with_vals = vals != nullptr;
    const int passes = (bits + 7) / 8;
    if (n == 0) return cudaSuccess;
    if (passes == 0 || n == 1) {
        // nothing to order: the words (and row ids) in input order
        if (pack) {
            const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, RS_THREADS), (int64_t)c.num_sms * 16));
            k_pack_words<<<grid, RS_THREADS, 0, c.stream>>>(*pack, n, keys, vals); c.launches++;
            GJ_CUDA_TRY(cudaGetLastError());
        }
        return cudaSuccess;
    }
    const size_t smem = with_vals ? RS_SMEM : RS_SMEM_K;
    if (with_vals) {
        GJ_CUDA_TRY(cudaFuncSetAttribute(k_onesweep_t<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        GJ_CUDA_TRY(cudaFuncSetAttribute(k_onesweep_t<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    } else {
        GJ_CUDA_TRY(cudaFuncSetAttribute(k_onesweep_t<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        GJ_CUDA_TRY(cudaFuncSetAttribute(k_onesweep_t<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    const int64_t tiles = ceil_div(n, RS_TILE);
    uint32_t *hist = nullptr;
    unsigned long long *status = nullptr;
    Temps tmp(c);
    GJ_CUDA_TRY(tmp.alloc(&hist, RS_MAX_PASSES * RS_RADIX + RS_MAX_PASSES));
    GJ_CUDA_TRY(tmp.alloc(&status, (size_t)tiles * RS_RADIX));
    uint32_t *counters = hist + RS_MAX_PASSES * RS_RADIX;
    GJ_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (RS_MAX_PASSES * RS_RADIX + RS_MAX_PASSES), c.stream));
    const PackSrc ps = pack ? *pack : PackSrc{};
    int hist_blocks = (int)std::min<int64_t>(ceil_div(n, RS_THREADS * 16), (int64_t)c.num_sms * 8);
    if (hist_blocks < 1) hist_blocks = 1;
    if (pack)
        k_digit_hist<true><<<hist_blocks, RS_THREADS, 0, c.stream>>>(nullptr, ps, n, lo_bit, passes, hist);
    else
        k_digit_hist<false><<<hist_blocks, RS_THREADS, 0, c.stream>>>(keys, ps, n, lo_bit, passes, hist);
    c.launches++;
    k_hist_to_base<<<passes, RS_RADIX, 0, c.stream>>>(hist); c.launches++;
    uint64_t *ka = keys, *kb = alt;
    uint32_t *va = vals, *vb = valt;
    for (int p = 0; p < passes; p++) {
        unsigned long long *st = status;   // one pass's lookback state at a time
        GJ_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(unsigned long long) * tiles * RS_RADIX, c.stream));
        const int shift = lo_bit + 8 * p;
        // the first pass of a packed sort reads the columns and writes into
        // `alt`; later passes ping-pong
        if (with_vals) {
            if (p == 0 && pack)
                k_onesweep_t<true, true><<<(unsigned)tiles, RS_THREADS, smem, c.stream>>>(
                    nullptr, ps, nullptr, kb, vb, n, shift, hist + p * RS_RADIX, counters + p, st, c.err);
            else
                k_onesweep_t<true, false><<<(unsigned)tiles, RS_THREADS, smem, c.stream>>>(
                    ka, ps, va, kb, vb, n, shift, hist + p * RS_RADIX, counters + p, st, c.err);
        } else {
            if (p == 0 && pack)
                k_onesweep_t<false, true><<<(unsigned)tiles, RS_THREADS, smem, c.stream>>>(
                    nullptr, ps, nullptr, kb, nullptr, n, shift, hist + p * RS_RADIX, counters + p, st, c.err);
            else
                k_onesweep_t<false, false><<<(unsigned)tiles, RS_THREADS, smem, c.stream>>>(
                    ka, ps, nullptr, kb, nullptr, n, shift, hist + p * RS_RADIX, counters + p, st, c.err);
        }
        c.launches++;
        GJ_CUDA_TRY(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    *kres = ka;
    if (vres) *vres = va;
    return cudaSuccess;
}

}  // namespace gj

