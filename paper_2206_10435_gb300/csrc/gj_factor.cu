// gj_factor.cu -- factor construction (Section 3.2, quantitative learning).
//
// A relation's potential is its exact frequency table: the distinct key
// tuples with their counts.  Here it is built by sorting the rows by their
// key tuple and cutting the sorted order into groups:
//
//   1. per key column, min and max (one read of every column);
//   2. each column becomes an unsigned field of ceil(log2(max-min+1)) bits;
//      fields are packed into 64-bit words, most significant column first,
//      and the words are sorted least significant first with the stable
//      radix sort (one word suffices unless the fields exceed 64 bits);
//   3. group heads are the rows whose packed key differs from the previous
//      row's; an exclusive scan numbers the groups;
//   4. each group records its first position and its key values; payload
//      columns are gathered into group order.
//
// Sorted order is also the order the desummariser walks: groups sharing a
// separator value are contiguous (the separator columns lead the order) and
// inside a group rows keep increasing row id.
#include <algorithm>

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
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT) {
        int32_t v = col[i];
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

// head[i]: the two-word key (hi, lo) differs from the previous one
__global__ void k_heads_packed2(const uint64_t *__restrict__ hi, const uint64_t *__restrict__ lo,
                                int64_t n, uint8_t *head) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT)
        head[i] = (i == 0) || hi[i] != hi[i - 1] || lo[i] != lo[i - 1];
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

// group starts and key values from the sorted packed keys (no random reads
// of the key columns)
__global__ void k_group_compact_packed(UnpackSpec u, const uint64_t *__restrict__ keys,
                                       const uint64_t *__restrict__ keys_hi,
                                       const uint32_t *__restrict__ perm,
                                       const uint8_t *__restrict__ head,
                                       const uint32_t *__restrict__ gid, int64_t n, int64_t G,
                                       uint32_t *gstart, int32_t *gkey) {
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT) {
        if (!head[i]) continue;
        const uint32_t g = gid[i];
        gstart[g] = (uint32_t)i;
        const uint64_t klo = keys[i], khi = keys_hi ? keys_hi[i] : 0ull;
        for (int c = 0; c < u.ncol; c++) {
            const uint64_t k = u.hi[c] ? khi : klo;
            const uint64_t mask = u.bits[c] >= 32 ? 0xFFFFFFFFull : ((1ull << u.bits[c]) - 1);
            const uint32_t v = (u.shift[c] < 64 ? (uint32_t)((k >> u.shift[c]) & mask) : 0u) + (uint32_t)u.mn[c];
            gkey[(int64_t)u.col[c] * G + g] = (int32_t)v;
        }
        if (u.nother) {
            const uint32_t r = perm[i];
            for (int c = 0; c < u.nother; c++) gkey[(int64_t)u.other_col[c] * G + g] = u.other[c][r];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) gstart[G] = (uint32_t)n;
}

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
        GJ_CUDA_TRY(dalloc(c, &mm, 2 * R.nk));
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
        dfree(c, mm);
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

// One factor build in two stages, so that the builds of several relations
// share their host synchronisations: the key ranges (for the packed field
// widths) before the sort, and the group counts (for the group arrays)
// after it.
struct FactorBuild {
    Relation *R = nullptr;
    Factor *F = nullptr;
    std::vector<int> bits;
    std::vector<std::vector<int>> words;
    uint64_t *keys = nullptr;      // the (low) packed word, in sorted order
    uint64_t *keys_hi = nullptr;   // a two-word key's high word, in sorted order
    uint64_t *lo = nullptr;        // two-word key: the low word, moved to the final order
    uint32_t *pos = nullptr, *perm = nullptr;
    uint8_t *head = nullptr;
    uint32_t *gid = nullptr, *gcount = nullptr;
    int32_t *sorted = nullptr;
};

void fb_free(Ctx &c, FactorBuild &b) {
    dfree(c, b.keys);
    dfree(c, b.keys_hi);
    dfree(c, b.lo);
    dfree(c, b.pos);
    dfree(c, b.perm);
    dfree(c, b.head);
    dfree(c, b.gid);
    dfree(c, b.gcount);
    dfree(c, b.sorted);
}

// stage 1 (key ranges known): rows sorted by the key tuple, group heads
// marked and numbered; the group count lands in b.gcount
cudaError_t fb_sort(Ctx &c, FactorBuild &b) {
    Relation &R = *b.R;
    Factor &F = *b.F;
    const std::vector<int> &order = F.order;
    F.n = R.n;
    const int64_t n = R.n;
    GJ_CUDA_TRY(dalloc(c, &F.perm, n));
    if (n == 0) return cudaSuccess;
    // field widths, least significant column last in `order`
    std::vector<int> &bits = b.bits;
    bits.assign(R.nk, 0);
    for (int i = 0; i < R.nk; i++)
        bits[i] = bits_of((uint32_t)((int64_t)R.kmax[i] - (int64_t)R.kmin[i]));
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
    GJ_CUDA_TRY(dalloc(c, &b.keys, n));
    // A two-word key sorts its high word carrying positions in the low
    // word's sorted order instead of row ids: one gather then brings the row
    // ids and the low word into the final order, and the groups are found
    // and unpacked from the two words (no re-read of the key columns).
    const bool two = words.size() == 2;
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
        if (two && w == 1) {
            GJ_CUDA_TRY(dalloc(c, &b.keys_hi, n));
            GJ_CUDA_TRY(dalloc(c, &b.pos, n));
            k_pack_pos<<<grid_for(c, n), FT, 0, c.stream>>>(ps, F.perm, n, b.keys_hi, b.pos); c.launches++;
            GJ_CUDA_TRY(cudaGetLastError());
            GJ_CUDA_TRY(radix_sort_u64_u32(c, b.keys_hi, b.pos, n, shift));
            GJ_CUDA_TRY(dalloc(c, &b.lo, n));
            GJ_CUDA_TRY(dalloc(c, &b.perm, n));
            k_compose<<<grid_for(c, n), FT, 0, c.stream>>>(b.pos, F.perm, b.keys, n, b.perm, b.lo); c.launches++;
            GJ_CUDA_TRY(cudaGetLastError());
            std::swap(F.perm, b.perm);
            std::swap(b.keys, b.lo);
            dfree(c, b.perm);
            dfree(c, b.lo);
            dfree(c, b.pos);
        } else {
            k_pack<<<grid_for(c, n), FT, 0, c.stream>>>(ps, w == 0 ? nullptr : F.perm, n, b.keys, F.perm); c.launches++;
            GJ_CUDA_TRY(cudaGetLastError());
            GJ_CUDA_TRY(radix_sort_u64_u32(c, b.keys, F.perm, n, shift));
        }
    }
    uint64_t *keys = b.keys;
    GJ_CUDA_TRY(dalloc(c, &b.head, n));
    GJ_CUDA_TRY(dalloc(c, &b.gid, n));
    GJ_CUDA_TRY(dalloc(c, &b.gcount, 1));
    uint8_t *head = b.head;
    uint32_t *gid = b.gid, *gcount = b.gcount;
    ColSet all{};
    all.ncol = R.nk;
    for (int i = 0; i < R.nk; i++) all.col[i] = R.key[i];
    int32_t *&sorted = b.sorted;
    if (words.size() == 1) {
        k_heads_packed<<<grid_for(c, n), FT, 0, c.stream>>>(keys, n, head); c.launches++;
    } else if (two) {
        k_heads_packed2<<<grid_for(c, n), FT, 0, c.stream>>>(b.keys_hi, keys, n, head); c.launches++;
    } else {
        // the key spans more than two words: bring the columns into sorted order
        // once, then find heads and groups with sequential reads
        GJ_CUDA_TRY(dalloc(c, &sorted, (size_t)R.nk * n));
        k_gather_cols<<<grid_for(c, n), FT, 0, c.stream>>>(all, F.perm, n, sorted); c.launches++;
        ColIdx by{};
        by.n = (int)order.size();
        for (int i = 0; i < by.n; i++) by.idx[i] = order[i];
        k_heads_sorted<<<grid_for(c, n), FT, 0, c.stream>>>(sorted, by, n, head); c.launches++;
    }
    GJ_CUDA_TRY(cudaGetLastError());
    GJ_CUDA_TRY(scan_u32(c, nullptr, head, gid, n, gcount));
    return cudaSuccess;
}

// stage 2 (group count G known): group starts and keys, payloads in group
// order; frees the stage's temporaries
cudaError_t fb_groups(Ctx &c, FactorBuild &b, int64_t G) {
    Relation &R = *b.R;
    Factor &F = *b.F;
    const std::vector<int> &order = F.order;
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
    const std::vector<int> &bits = b.bits;
    const std::vector<std::vector<int>> &words = b.words;
    uint64_t *keys = b.keys;
    uint8_t *head = b.head;
    uint32_t *gid = b.gid;
    int32_t *&sorted = b.sorted;
    F.G = G;
    GJ_CUDA_TRY(dalloc(c, &F.gstart, F.G + 1));
    GJ_CUDA_TRY(dalloc(c, &F.gkey, (size_t)R.nk * F.G));
    if (sorted) {
        k_group_compact_sorted<<<grid_for(c, n), FT, 0, c.stream>>>(sorted, R.nk, head, gid, n, F.G,
                                                                    F.gstart, F.gkey); c.launches++;
        dfree(c, sorted);
    } else {
        // one or two packed words: unpack the key values of every group head
        UnpackSpec u{};
        for (size_t w = 0; w < words.size(); w++) {
            int shift = 0;
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
        k_group_compact_packed<<<grid_for(c, n), FT, 0, c.stream>>>(u, keys, b.keys_hi, F.perm, head, gid, n,
                                                                    F.G, F.gstart, F.gkey); c.launches++;
    }
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
    if (words_mm * 4 > (1 << 16) || m * 4 > (1 << 16)) return cudaErrorInvalidValue;
    if (words_mm) {
        int32_t *mm = nullptr;
        GJ_CUDA_TRY(dalloc(c, &mm, words_mm));
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
        dfree(c, mm);
    }
    std::vector<FactorBuild> b(m);
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < m && e == cudaSuccess; i++) {
        b[i].R = R[i];
        b[i].F = F[i];
        e = fb_sort(c, b[i]);
    }
    // group counts, one readback
    uint32_t *hg = (uint32_t *)c.pinned;
    for (size_t i = 0; i < m && e == cudaSuccess; i++)
        if (b[i].gcount) e = cudaMemcpyAsync(hg + i, b[i].gcount, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    std::vector<int64_t> G(m, 0);
    if (e == cudaSuccess)
        for (size_t i = 0; i < m; i++) G[i] = b[i].gcount ? (int64_t)hg[i] : 0;
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
