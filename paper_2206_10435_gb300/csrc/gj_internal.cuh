// gj_internal.cuh -- shared definitions of the CUDA path (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "gj.h"

namespace gj {

// ------------------------------------------------------------------ semiring
// Counting semiring over N with a saturation marker SAT = 2^64 - 1 that
// stands for "2^64 - 1 or more".  0 annihilates SAT, so a dead branch of the
// join tree stays 0 however large the counts beneath it.

constexpr uint64_t SAT = ~0ull;
constexpr uint32_t NONE = 0xFFFFFFFFu;

__host__ __device__ __forceinline__ uint64_t sat_add(uint64_t a, uint64_t b) {
    uint64_t s = a + b;
    return (s < a || s == SAT) ? SAT : s;
}

__device__ __forceinline__ uint64_t sat_mul(uint64_t a, uint64_t b) {
    if (a == 0 || b == 0) return 0;
    uint64_t hi = __umul64hi(a, b);
    uint64_t lo = a * b;
    return (hi != 0 || lo == SAT) ? SAT : lo;
}

// ------------------------------------------------------------------ errors
// Device-side error word: kernels OR these bits in instead of trapping.
enum : uint32_t {
    ERRF_TIMEOUT = 1u,   // a bounded spin-wait gave up
    ERRF_BOUNDS = 2u,    // an index check failed
    ERRF_OVERFLOW = 4u,  // a count that must be exact saturated
};

// Upper bound on polls of a lookback flag before a kernel gives up.
constexpr uint32_t SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ void raise_err(uint32_t *err, uint32_t bits) {
    if (err) atomicOr(err, bits);
}

// ------------------------------------------------------------------ context
struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    // stream-ordered pool owned by the context; it keeps freed memory for
    // reuse instead of returning it to the CUDA driver at every synchronisation
    cudaMemPool_t pool = nullptr;
    uint32_t *err = nullptr;          // device error word
    uint64_t *pinned = nullptr;       // small pinned host buffer for readbacks
    int num_sms = 0;
    uint64_t launches = 0;            // kernels launched (profiling)
    int emit_rpt = 4;                 // result rows per thread of the emit kernel (2, 4 or 8)
    int tri_mode = 0;                 // triangle intersection: 0 chooses, 1 sorted lists, 2 bitmaps
    int down_combine = 0;             // downward pass: 0 by key order, 1 never, 2 always
    size_t slot_arena = (size_t)512 << 20;   // arena bytes of each server slot
    // failure injection (tests): polls before the group scan's bounded wait
    // gives up, whether tile 0 of that scan withholds its status (so the
    // wait runs out), and the stream-ordered allocation to fail (counted
    // from when the option was set; 0 = none)
    uint32_t spin_limit = SPIN_LIMIT;
    bool test_stall = false;
    int64_t fail_alloc_at = 0;
    int64_t allocs = 0;
    // bump arena (a serving slot's): while arena_on, allocations come from
    // it as long as it has room, and frees of its memory are no-ops; the
    // owner rewinds arena_used once nothing enqueued later on this stream
    // needs what lies past the mark (the stream orders reuse)
    char *arena = nullptr;
    size_t arena_size = 0, arena_used = 0;
    bool arena_on = false;
    // device-time profile of the emit kernel (CUDA events on the stream)
    bool prof = false;
    std::vector<cudaEvent_t> ev_free, ev_used;     // emit kernel: start/stop pairs
    std::vector<cudaEvent_t> xev_used;             // window expansion: start/stop pairs
    uint64_t emit_launches = 0, emit_rows = 0, emit_bytes = 0;
    cudaEvent_t event(bool expansion = false) {
        cudaEvent_t e = nullptr;
        if (!ev_free.empty()) { e = ev_free.back(); ev_free.pop_back(); }
        else cudaEventCreate(&e);
        (expansion ? xev_used : ev_used).push_back(e);
        return e;
    }
};

// Stream-ordered device allocation on the context's stream.
// An allocation the failure-injection option makes fail.
inline bool fail_this_alloc(Ctx &c) {
    c.allocs++;
    return c.fail_alloc_at > 0 && c.allocs == c.fail_alloc_at;
}

inline bool in_arena(const Ctx &c, const void *p) {
    return c.arena && (const char *)p >= c.arena && (const char *)p < c.arena + c.arena_size;
}

// bytes from the arena (256-byte aligned), or NULL
inline void *arena_take(Ctx &c, size_t bytes) {
    if (!c.arena_on) return nullptr;
    const size_t b = (bytes + 255) & ~(size_t)255;
    if (b > c.arena_size - c.arena_used) return nullptr;
    void *p = c.arena + c.arena_used;
    c.arena_used += b;
    return p;
}

inline cudaError_t dalloc_bytes(Ctx &c, void **p, size_t bytes) {
    *p = nullptr;
    if (fail_this_alloc(c)) return cudaErrorMemoryAllocation;
    if (bytes == 0) bytes = 1;
    if ((*p = arena_take(c, bytes)) != nullptr) return cudaSuccess;
    if (c.pool) return cudaMallocFromPoolAsync(p, bytes, c.pool, c.stream);
    return cudaMallocAsync(p, bytes, c.stream);
}
template <class T>
inline cudaError_t dalloc(Ctx &c, T **p, size_t count) {
    return dalloc_bytes(c, (void **)p, (count == 0 ? 1 : count) * sizeof(T));
}
inline void dfree_bytes(Ctx &c, void *p) {
    if (p && !in_arena(c, p)) cudaFreeAsync(p, c.stream);
}
template <class T>
inline void dfree(Ctx &c, T *&p) {
    dfree_bytes(c, (void *)p);
    p = nullptr;
}

// Stream-ordered temporaries of one scope: freed when the scope ends, on
// every path out of it (an error return included).  keep() hands one over
// to a longer-lived owner.
class Temps {
  public:
    explicit Temps(Ctx &c) : c_(c) {}
    Temps(const Temps &) = delete;
    Temps &operator=(const Temps &) = delete;
    ~Temps() {
        for (void *p : p_) dfree_bytes(c_, p);
    }
    template <class T>
    cudaError_t alloc(T **p, size_t count) {
        cudaError_t e = dalloc(c_, p, count);
        if (e == cudaSuccess) p_.push_back((void *)*p);
        return e;
    }
    cudaError_t alloc_bytes(void **p, size_t bytes) {
        cudaError_t e = dalloc_bytes(c_, p, bytes);
        if (e == cudaSuccess) p_.push_back(*p);
        return e;
    }
    void keep(const void *p) {
        for (size_t i = 0; i < p_.size(); i++)
            if (p_[i] == p) { p_.erase(p_.begin() + i); return; }
    }
    // frees p now (it must be one of these temporaries)
    template <class T>
    void free(T *&p) {
        keep((const void *)p);
        dfree(c_, p);
    }

  private:
    Ctx &c_;
    std::vector<void *> p_;
};

// ------------------------------------------------------------------ primitives
// Exclusive prefix sums, single pass with decoupled lookback.  All of them
// are stream-ordered; *total_dev (if non-NULL) receives the sum.

// u32: out[i] = sum of in[0..i); in may be NULL with flags != NULL, in which
// case the summed value of i is (flags[i] != 0).
cudaError_t scan_u32(Ctx &c, const uint32_t *in, const uint8_t *flags, uint32_t *out,
                     int64_t n, uint32_t *total_dev);

// scan_u32 over the first *n_dev elements (a count in device memory) of
// arrays sized for `cap`; *total_dev may alias nothing else.  No host sync.
cudaError_t scan_u32_dev(Ctx &c, const uint32_t *in, const uint8_t *flags, uint32_t *out,
                         int64_t cap, const uint32_t *n_dev, uint32_t *total_dev);

// saturating u64, optionally segmented: heads[i] != 0 starts a new segment
// (the exclusive value there is 0).  seg_total[s] (if non-NULL) receives the
// saturating sum of segment s, with seg_id[i] mapping element i to its
// segment (needed only when seg_total is set); total_dev gets the sum of the
// last segment (or of everything, unsegmented).
cudaError_t scan_u64_sat(Ctx &c, const uint64_t *in, const uint8_t *heads, uint64_t *out,
                         int64_t n, uint64_t *total_dev, uint64_t *seg_total,
                         const uint32_t *seg_id);

// Key columns packed into one 64-bit word: field c is (col[c][i] - mn[c])
// at bit shift[c] (a field at shift >= 64 has no bits and is left out);
// with row_bits > 0 the row id i fills the low row_bits bits, under the key.
constexpr int PACK_MAX_COLS = 8;
struct PackSrc {
    int ncol;
    const int32_t *col[PACK_MAX_COLS];
    int32_t mn[PACK_MAX_COLS];
    int shift[PACK_MAX_COLS];
    int row_bits;
};

__device__ __forceinline__ uint64_t pack_word(const PackSrc &ps, int64_t i) {
    uint64_t k = ps.row_bits ? (uint64_t)i : 0ull;
#pragma unroll
    for (int c = 0; c < PACK_MAX_COLS; c++)
        if (c < ps.ncol && ps.shift[c] < 64)
            k |= (uint64_t)((uint32_t)__ldg(ps.col[c] + i) - (uint32_t)ps.mn[c]) << ps.shift[c];
    return k;
}

// Stable LSD radix sort of 64-bit words on bits [lo_bit, lo_bit + bits),
// 8 bits per pass.  The words are `pack` applied to rows 0..n-1 when pack is
// non-NULL (the words are then built by the first pass and never read from
// memory; `keys` is only a buffer), else keys[0..n).  With vals (non-NULL)
// each word carries a 32-bit value: the row id when packing, else vals[i].
// The passes ping-pong between keys/alt (and vals/valt); *kres and *vres
// receive the buffers holding the sorted result.  Buffers hold n entries.
cudaError_t radix_sort_words(Ctx &c, const PackSrc *pack, uint64_t *keys, uint64_t *alt,
                             uint32_t *vals, uint32_t *valt, int64_t n, int lo_bit, int bits,
                             uint64_t **kres, uint32_t **vres);

// Stable LSD radix sort of (key, value) pairs on key bits [0, bits).
// keys/vals are sorted in place (ping-pong through internal buffers).
cudaError_t radix_sort_u64_u32(Ctx &c, uint64_t *keys, uint32_t *vals, int64_t n, int bits);

// Tile sizes of the radix sort and of the 32-bit scans: callers that lay out
// the sort's status words or a scan's lookback state themselves (the
// allocation-free factor build) size them from these.
constexpr int RADIX_SORT_TILE = 256 * 16;   // keys per onesweep tile
constexpr int RADIX_SORT_BINS = 256;        // digit values per pass
constexpr int RADIX_SORT_MAX_PASSES = 8;
constexpr int SCAN_U32_TILE = 256 * 16;     // elements per 32-bit scan tile

// Bytes of lookback state scan_u32_in needs for n elements.
constexpr size_t scan_u32_state_bytes_for(int64_t n) {
    return 16 + ((((size_t)((n > 0 ? n : 1) + SCAN_U32_TILE - 1) / SCAN_U32_TILE) * 4 + 15) & ~(size_t)15) +
           2 * (size_t)(((n > 0 ? n : 1) + SCAN_U32_TILE - 1) / SCAN_U32_TILE) * sizeof(uint32_t);
}

// ------------------------------------------------------------------ helpers
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Records the failing CUDA call (error name, file, line) for gj_last_error.
void note_cuda_error(cudaError_t e, const char *file, int line);

#define GJ_CUDA_TRY(expr)                                        \
    do {                                                         \
        cudaError_t _e = (expr);                                 \
        if (_e != cudaSuccess) {                                 \
            ::gj::note_cuda_error(_e, __FILE__, __LINE__);       \
            return _e;                                           \
        }                                                        \
    } while (0)

}  // namespace gj
