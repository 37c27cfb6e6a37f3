// gj_emit.cu -- desummarisation, the emit step (Section 3.6).
//
// Emission with RPT (2 or 4) consecutive rows per thread.  The thread finds the block
// of its first row by a search of the staged block offsets and splits that
// row's offset into per-relation digits once; the next rows follow by
// incrementing the digits like an odometer (rows of a block are ordered
// r_1..r_k, relation k fastest), stepping to the next block when the
// odometer wraps.  Output columns are grouped by the relation they come
// from, so the group and position of that relation are compile-time
// register indices.  Each column is written through a per-warp
// shared-memory transpose so that every store instruction covers 32
// consecutive rows of the column (streaming stores: the result is not
// read back by this kernel).
#include <algorithm>

#include "gj_emit.cuh"

namespace gj {
namespace {

// tile_first[t] = block holding the first row of emit tile t (rows
// [row0 + t*tile_rows, ...)): the last block whose first row is <= that
// row, by a binary search of the block offsets per tile (a window has far
// fewer tiles than blocks, and the top levels of the searches stay in
// cache).
__global__ void k_tile_first(const uint64_t *__restrict__ A, const uint32_t *B_dev, uint64_t row0,
                             int64_t tiles, int64_t tile_rows, uint32_t *tile_first) {
    const int64_t B = *B_dev;
    for (int64_t t = (int64_t)blockIdx.x * EMIT_DT + threadIdx.x; t < tiles; t += (int64_t)gridDim.x * EMIT_DT) {
        const uint64_t row = row0 + (uint64_t)(t * tile_rows);
        int64_t lo = 0, hi = B;   // first block whose first row is > row
        while (lo < hi) {
            const int64_t m = (lo + hi) >> 1;
            if (A[m] <= row) lo = m + 1; else hi = m;
        }
        tile_first[t] = (uint32_t)(lo > 0 ? lo - 1 : 0);
    }
}

// Column stores.  A lane holds RPT consecutive rows of a column.  Every
// store writes a whole 32-byte sector: the G = 32 / (RPT * sizeof(T)) lanes
// of a group pass their values to the group's first lane by shuffle, and
// that lane writes the group's 32 consecutive bytes with one vector store
// (v4.b64 or v8.b32).  Edges of the window (or unaligned buffers) fall back
// to scalar stores.  Streaming (.cs) stores: the result is not read here.
__device__ __forceinline__ void st_cs_32B(unsigned long long *p, const unsigned long long (&v)[4]) {
    asm volatile("st.global.cs.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(v[0]), "l"(v[1]),
                 "l"(v[2]), "l"(v[3]) : "memory");
}

__device__ __forceinline__ void st_cs_32B(unsigned int *p, const unsigned int (&v)[8]) {
    asm volatile("st.global.cs.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                 "r"(v[7]) : "memory");
}

// Loads with an L2 eviction priority (createpolicy + L2::cache_hint): the
// factors' arrays (group starts, keys, payloads, row ids) are gathered
// again and again and should stay in L2; the block list is read once and
// should leave first, as should the result columns (streaming stores).
__device__ __forceinline__ uint64_t policy_keep() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_once() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned int ld_hint(const unsigned int *a, uint64_t pol) {
    unsigned int v;
    asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ int ld_hint(const int *a, uint64_t pol) {
    return (int)ld_hint((const unsigned int *)a, pol);
}
__device__ __forceinline__ unsigned long long ld_hint(const unsigned long long *a, uint64_t pol) {
    unsigned long long v;
    asm("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(a), "l"(pol));
    return v;
}

// all lanes of the warp must call this (shuffles)
template <int RPT, class T>
__device__ __forceinline__ void emit_store_col(const T (&v)[RPT], T *dst, int64_t rbeg, int nrow,
                                               int group_rows, bool vec, int lane) {
    constexpr int PER = 32 / (int)sizeof(T);   // values in one 32-byte store
    if constexpr (RPT >= PER) {
        // the lane's own rows fill whole sectors
        static_assert(RPT % PER == 0, "rows per thread must fill whole sectors");
        if (vec && nrow == RPT) {
#pragma unroll
            for (int s = 0; s < RPT / PER; s++) {
                T part[PER];
#pragma unroll
                for (int i = 0; i < PER; i++) part[i] = v[s * PER + i];
                st_cs_32B(dst + rbeg + s * PER, part);
            }
        } else {
#pragma unroll
            for (int i = 0; i < RPT; i++)
                if (i < nrow) __stcs(dst + rbeg + i, v[i]);
        }
    } else {
        constexpr int G = PER / RPT;           // lanes per 32-byte group
        static_assert(G * RPT == PER, "rows per thread must divide a sector");
        T all[PER];
#pragma unroll
        for (int i = 0; i < RPT; i++) all[i] = v[i];
#pragma unroll
        for (int k = 1; k < G; k++)
#pragma unroll
            for (int i = 0; i < RPT; i++) all[k * RPT + i] = __shfl_down_sync(0xffffffffu, v[i], k);
        if (vec && group_rows == PER) {
            if ((lane & (G - 1)) == 0) st_cs_32B(dst + rbeg, all);
        } else {
#pragma unroll
            for (int i = 0; i < RPT; i++)
                if (i < nrow) __stcs(dst + rbeg + i, v[i]);
        }
    }
}

template <int K, int RPT>
__global__ void __launch_bounds__(EMIT_DT, (RPT == 8 ? 2 : RPT == 4 ? (K <= 3 ? 5 : K <= 5 ? 4 : 3) : (K <= 5 ? 6 : 4)))
k_emit(Emit4Spec e, const uint32_t *__restrict__ tile_first, int64_t tiles, const uint32_t *B_dev,
       uint64_t row0, int64_t n) {
    constexpr int TILE = EMIT_DT * RPT;
    const int64_t B = *B_dev;
    __shared__ uint64_t s_A[TILE + 1];
    const int64_t tile = blockIdx.x;
    const int64_t r0 = tile * TILE;
    if (r0 >= n) return;
    const int64_t r1 = min(n, r0 + TILE);
    const int64_t first = tile_first[tile];
    const int64_t last = (tile + 1 < tiles) ? (int64_t)tile_first[tile + 1] : B - 1;
    int nb = (int)(last - first + 1);
    // the tile's rows plus the block holding the next tile's first row
    if (last < first || nb > TILE + 1) {   // cannot happen: every block has >= 1 row
        if (threadIdx.x == 0) raise_err(e.err, ERRF_BOUNDS);
        return;
    }
    const uint64_t keep = policy_keep(), once = policy_once();
    for (int t = threadIdx.x; t < nb; t += EMIT_DT)
        s_A[t] = ld_hint((const unsigned long long *)e.A + first + t, once);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t rbeg = r0 + (int64_t)threadIdx.x * RPT;
    // lanes past the end still take part in the warp's shuffles
    const int nrow = (int)max((int64_t)0, min((int64_t)RPT, r1 - rbeg));
    // rows of a 32-byte store group of 32-bit and of 64-bit columns
    const int g32 = (int)max((int64_t)0, min((int64_t)8, r1 - (rbeg & ~(int64_t)7)));
    const int g64 = (int)max((int64_t)0, min((int64_t)4, r1 - (rbeg & ~(int64_t)3)));
    const uint64_t row = row0 + (uint64_t)rbeg;
    // block of every row: a search for the first, then at most one step per row
    int lb[RPT];
    if (nrow > 0) {
        int a = 0, b = nb;
        while (a < b) { int m = (a + b) >> 1; if (s_A[m] <= row) a = m + 1; else b = m; }
        lb[0] = a - 1;
    } else {
        lb[0] = 0;
    }
#pragma unroll
    for (int i = 1; i < RPT; i++) {
        lb[i] = lb[i - 1];
        if (i < nrow && lb[i] + 1 < nb && s_A[lb[i] + 1] <= row + i) lb[i]++;
    }
    const uint64_t q0 = nrow > 0 ? row - s_A[lb[0]] : 0;
    // all group ids, then all group extents: two rounds of independent loads;
    // a row in the same block as the previous row reuses its values (the
    // load is predicated off, so it costs no memory traffic)
    bool nb_row[RPT];
#pragma unroll
    for (int i = 0; i < RPT; i++) nb_row[i] = (i == 0) || lb[i] != lb[i - 1];
    uint32_t g[RPT][K];
#pragma unroll
    for (int i = 0; i < RPT; i++)
#pragma unroll
        for (int j = 0; j < K; j++)
            g[i][j] = nb_row[i] ? ld_hint(e.grp[j] + first + lb[i], once) : g[i > 0 ? i - 1 : 0][j];
    // key columns need only the groups: write them while extents load
#pragma unroll
    for (int j = 0; j < K; j++) {
        for (int c = e.col_off[j]; c < e.col_off[j + 1]; c++) {
            if (e.kind[c] != 0) continue;
            const unsigned int *src = (const unsigned int *)e.src[c];
            unsigned int v[RPT];
#pragma unroll
            for (int i = 0; i < RPT; i++)
                v[i] = nb_row[i] ? ld_hint(src + g[i][j], keep) : v[i > 0 ? i - 1 : 0];
            emit_store_col<RPT>(v, (unsigned int *)e.dst[c], rbeg, nrow, g32, e.vec, lane);
        }
    }
    uint32_t pos[RPT][K];
    {
        uint32_t base[RPT][K], cnt[RPT][K];
#pragma unroll
        for (int i = 0; i < RPT; i++)
#pragma unroll
            for (int j = 0; j < K; j++) {
                if (nb_row[i]) {
                    base[i][j] = ld_hint(e.gstart[j] + g[i][j], keep);
                    cnt[i][j] = ld_hint(e.gstart[j] + g[i][j] + 1, keep) - base[i][j];
                } else {
                    base[i][j] = base[i > 0 ? i - 1 : 0][j];
                    cnt[i][j] = cnt[i > 0 ? i - 1 : 0][j];
                }
            }
        // digits of the first row (relation k-1 fastest), then an odometer
        uint32_t d[K];
        uint64_t q = q0;
#pragma unroll
        for (int j = K - 1; j >= 0; j--) {
            uint32_t cj = cnt[0][j];
            if (cj <= 1) { d[j] = 0; continue; }
            if (q < 0x100000000ull) {
                uint32_t q32 = (uint32_t)q;
                d[j] = q32 % cj;
                q = q32 / cj;
            } else {
                d[j] = (uint32_t)(q % cj);
                q /= cj;
            }
        }
#pragma unroll
        for (int j = 0; j < K; j++) pos[0][j] = base[0][j] + d[j];
#pragma unroll
        for (int i = 1; i < RPT; i++) {
            if (lb[i] != lb[i - 1]) {
#pragma unroll
                for (int j = 0; j < K; j++) d[j] = 0;   // a block starts at digits 0
            } else {
                bool carry = true;
#pragma unroll
                for (int j = K - 1; j >= 0; j--) {
                    if (carry) {
                        d[j]++;
                        carry = d[j] >= cnt[i][j];
                        if (carry) d[j] = 0;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < K; j++) pos[i][j] = base[i][j] + d[j];
        }
    }
#pragma unroll
    for (int j = 0; j < K; j++) {
        for (int c = e.col_off[j]; c < e.col_off[j + 1]; c++) {
            const int kind = e.kind[c];
            if (kind == 2) {
                const unsigned long long *src = (const unsigned long long *)e.src[c];
                unsigned long long v[RPT];
#pragma unroll
                for (int i = 0; i < RPT; i++) v[i] = ld_hint(src + pos[i][j], keep);
                emit_store_col<RPT>(v, (unsigned long long *)e.dst[c], rbeg, nrow, g64, e.vec, lane);
            } else if (kind == 1) {
                const unsigned int *src = (const unsigned int *)e.src[c];
                unsigned int v[RPT];
#pragma unroll
                for (int i = 0; i < RPT; i++) v[i] = ld_hint(src + pos[i][j], keep);
                emit_store_col<RPT>(v, (unsigned int *)e.dst[c], rbeg, nrow, g32, e.vec, lane);
            }
        }
        if (e.rid_out[j]) {
            unsigned int v[RPT];
#pragma unroll
            for (int i = 0; i < RPT; i++) v[i] = ld_hint(e.perm[j] + pos[i][j], keep);
            emit_store_col<RPT>(v, e.rid_out[j], rbeg, nrow, g32,
                                e.vec && ((uintptr_t)e.rid_out[j] & 31) == 0, lane);
        }
    }
}

template <int K, int RPT>
cudaError_t launch_k(Ctx &c, const Emit4Spec &s, const uint32_t *B_dev, uint64_t row0, int64_t n,
                     const uint32_t *pre) {
    constexpr int TILE = EMIT_DT * RPT;
    const int64_t tiles = ceil_div(n, TILE);
    uint32_t *tile_first = nullptr;
    if (!pre) {
        GJ_CUDA_TRY(dalloc(c, &tile_first, tiles + 1));
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(tiles, EMIT_DT), (int64_t)c.num_sms * 16));
        k_tile_first<<<(unsigned)grid, EMIT_DT, 0, c.stream>>>(s.A, B_dev, row0, tiles, TILE, tile_first); c.launches++;
    }
    if (c.prof) cudaEventRecord(c.event(), c.stream);
    k_emit<K, RPT><<<(unsigned)tiles, EMIT_DT, 0, c.stream>>>(s, pre ? pre : tile_first, tiles, B_dev, row0, n); c.launches++;
    cudaError_t e = cudaGetLastError();
    dfree(c, tile_first);
    return e;
}

template <int RPT>
cudaError_t launch_rpt(Ctx &c, int k, const Emit4Spec &s, const uint32_t *B_dev, uint64_t row0,
                       int64_t n, const uint32_t *pre) {
    switch (k) {
        case 1: return launch_k<1, RPT>(c, s, B_dev, row0, n, pre);
        case 2: return launch_k<2, RPT>(c, s, B_dev, row0, n, pre);
        case 3: return launch_k<3, RPT>(c, s, B_dev, row0, n, pre);
        case 4: return launch_k<4, RPT>(c, s, B_dev, row0, n, pre);
        case 5: return launch_k<5, RPT>(c, s, B_dev, row0, n, pre);
        case 6: return launch_k<6, RPT>(c, s, B_dev, row0, n, pre);
        case 7: return launch_k<7, RPT>(c, s, B_dev, row0, n, pre);
        case 8: return launch_k<8, RPT>(c, s, B_dev, row0, n, pre);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_emit(Ctx &c, int k, const Emit4Spec &s, const uint32_t *B_dev, uint64_t row0,
                        int64_t n, const uint32_t *tile_first) {
    if (c.emit_rpt == 2) return launch_rpt<2>(c, k, s, B_dev, row0, n, tile_first);
    if (c.emit_rpt == 8) return launch_rpt<8>(c, k, s, B_dev, row0, n, tile_first);
    return launch_rpt<4>(c, k, s, B_dev, row0, n, tile_first);
}

}  // namespace gj
