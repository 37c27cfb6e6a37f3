// gj_emit.cu -- desummarisation, the emit step (Section 3.6).
//
// Emission with 4 consecutive rows per thread.  The thread finds the block
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
// [row0 + t*T, ...)); written by the blocks themselves, one scatter pass.
__global__ void k_tile_first(const uint64_t *__restrict__ A, const uint32_t *B_dev, uint64_t row0,
                             int64_t n, int64_t tiles, uint32_t *tile_first) {
    const int64_t B = *B_dev;
    for (int64_t b = (int64_t)blockIdx.x * EMIT_DT + threadIdx.x; b < B; b += (int64_t)gridDim.x * EMIT_DT) {
        uint64_t lo = A[b] > row0 ? A[b] - row0 : 0;
        uint64_t hi = (b + 1 < B) ? A[b + 1] - row0 : (uint64_t)n;
        int64_t t0 = (int64_t)((lo + EMIT4_TILE - 1) / EMIT4_TILE);
        int64_t t1 = (int64_t)((hi + EMIT4_TILE - 1) / EMIT4_TILE);
        for (int64_t t = t0; t < t1 && t < tiles; t++) tile_first[t] = (uint32_t)b;
    }
}

// Column stores.  A lane holds 4 consecutive rows of a column.  Every store
// writes whole 32-byte sectors: a 64-bit column stores its 4 values as one
// 32-byte vector store; a 32-bit column pairs lanes (2m, 2m+1) by shuffle
// and lane 2m stores the pair's 8 consecutive values as one 32-byte vector
// store.  Edges of the window (or unaligned buffers) fall back to scalar
// stores.  Streaming (.cs) stores: the result is not read back here.
__device__ __forceinline__ void st_cs_v4_b64(unsigned long long *p, const unsigned long long (&v)[EMIT_RPT]) {
    asm volatile("st.global.cs.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(v[0]), "l"(v[1]),
                 "l"(v[2]), "l"(v[3]) : "memory");
}

__device__ __forceinline__ void st_cs_v8_b32(unsigned int *p, const unsigned int (&a)[EMIT_RPT],
                                             const unsigned int (&b)[EMIT_RPT]) {
    asm volatile("st.global.cs.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p),
                 "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]),
                 "r"(b[3]) : "memory");
}

__device__ __forceinline__ void emit_store_col(const unsigned long long (&v)[EMIT_RPT],
                                               unsigned long long *dst, int64_t rbeg, int nrow,
                                               bool vec) {
    if (vec && nrow == EMIT_RPT) {
        st_cs_v4_b64(dst + rbeg, v);
    } else {
#pragma unroll
        for (int i = 0; i < EMIT_RPT; i++)
            if (i < nrow) __stcs(dst + rbeg + i, v[i]);
    }
}

// all lanes of the warp must call this (shuffles)
__device__ __forceinline__ void emit_store_col(const unsigned int (&v)[EMIT_RPT], unsigned int *dst,
                                               int64_t rbeg, int nrow, int pair_rows, bool vec,
                                               int lane) {
    unsigned int o[EMIT_RPT];
#pragma unroll
    for (int i = 0; i < EMIT_RPT; i++) o[i] = __shfl_xor_sync(0xffffffffu, v[i], 1);
    if (vec && pair_rows == 2 * EMIT_RPT) {
        if ((lane & 1) == 0) st_cs_v8_b32(dst + rbeg, v, o);
    } else {
#pragma unroll
        for (int i = 0; i < EMIT_RPT; i++)
            if (i < nrow) __stcs(dst + rbeg + i, v[i]);
    }
}

template <int K>
__global__ void __launch_bounds__(EMIT_DT, (K <= 5 ? 4 : 3))
k_emit4(Emit4Spec e, const uint32_t *__restrict__ tile_first, int64_t tiles, const uint32_t *B_dev,
        uint64_t row0, int64_t n) {
    const int64_t B = *B_dev;
    __shared__ uint64_t s_A[EMIT4_TILE + 1];
    const int64_t tile = blockIdx.x;
    const int64_t r0 = tile * EMIT4_TILE;
    if (r0 >= n) return;
    const int64_t r1 = min(n, r0 + EMIT4_TILE);
    const int64_t first = tile_first[tile];
    const int64_t last = (tile + 1 < tiles) ? (int64_t)tile_first[tile + 1] : B - 1;
    int nb = (int)(last - first + 1);
    // the tile's rows plus the block holding the next tile's first row
    if (last < first || nb > EMIT4_TILE + 1) {   // cannot happen: every block has >= 1 row
        if (threadIdx.x == 0) raise_err(e.err, ERRF_BOUNDS);
        return;
    }
    for (int t = threadIdx.x; t < nb; t += EMIT_DT) s_A[t] = e.A[first + t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t rbeg = r0 + (int64_t)threadIdx.x * EMIT_RPT;
    // lanes past the end still take part in the warp's shuffles
    const int nrow = (int)max((int64_t)0, min((int64_t)EMIT_RPT, r1 - rbeg));
    // rows of the lane pair (2m, 2m+1) that lane 2m would store
    const int pair_rows = (int)max((int64_t)0, min((int64_t)2 * EMIT_RPT, r1 - (rbeg & ~(int64_t)(2 * EMIT_RPT - 1))));
    const uint64_t row = row0 + (uint64_t)rbeg;
    // block of every row: a search for the first, then at most one step per row
    int lb[EMIT_RPT];
    if (nrow > 0) {
        int a = 0, b = nb;
        while (a < b) { int m = (a + b) >> 1; if (s_A[m] <= row) a = m + 1; else b = m; }
        lb[0] = a - 1;
    } else {
        lb[0] = 0;
    }
#pragma unroll
    for (int i = 1; i < EMIT_RPT; i++) {
        lb[i] = lb[i - 1];
        if (i < nrow && lb[i] + 1 < nb && s_A[lb[i] + 1] <= row + i) lb[i]++;
    }
    const uint64_t q0 = nrow > 0 ? row - s_A[lb[0]] : 0;
    // all group ids, then all group extents: two rounds of independent loads;
    // a row in the same block as the previous row reuses its values (the
    // load is predicated off, so it costs no memory traffic)
    bool nb_row[EMIT_RPT];
#pragma unroll
    for (int i = 0; i < EMIT_RPT; i++) nb_row[i] = (i == 0) || lb[i] != lb[i - 1];
    uint32_t g[EMIT_RPT][K];
#pragma unroll
    for (int i = 0; i < EMIT_RPT; i++)
#pragma unroll
        for (int j = 0; j < K; j++)
            g[i][j] = nb_row[i] ? __ldg(e.grp[j] + first + lb[i]) : g[i > 0 ? i - 1 : 0][j];
    // key columns need only the groups: write them while extents load
#pragma unroll
    for (int j = 0; j < K; j++) {
        for (int c = e.col_off[j]; c < e.col_off[j + 1]; c++) {
            if (e.kind[c] != 0) continue;
            const unsigned int *src = (const unsigned int *)e.src[c];
            unsigned int v[EMIT_RPT];
#pragma unroll
            for (int i = 0; i < EMIT_RPT; i++)
                v[i] = nb_row[i] ? __ldg(src + g[i][j]) : v[i > 0 ? i - 1 : 0];
            emit_store_col(v, (unsigned int *)e.dst[c], rbeg, nrow, pair_rows, e.vec, lane);
        }
    }
    uint32_t pos[EMIT_RPT][K];
    {
        uint32_t base[EMIT_RPT][K], cnt[EMIT_RPT][K];
#pragma unroll
        for (int i = 0; i < EMIT_RPT; i++)
#pragma unroll
            for (int j = 0; j < K; j++) {
                if (nb_row[i]) {
                    base[i][j] = __ldg(e.gstart[j] + g[i][j]);
                    cnt[i][j] = __ldg(e.gstart[j] + g[i][j] + 1) - base[i][j];
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
        for (int i = 1; i < EMIT_RPT; i++) {
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
                unsigned long long v[EMIT_RPT];
#pragma unroll
                for (int i = 0; i < EMIT_RPT; i++) v[i] = __ldg(src + pos[i][j]);
                emit_store_col(v, (unsigned long long *)e.dst[c], rbeg, nrow, e.vec);
            } else if (kind == 1) {
                const unsigned int *src = (const unsigned int *)e.src[c];
                unsigned int v[EMIT_RPT];
#pragma unroll
                for (int i = 0; i < EMIT_RPT; i++) v[i] = __ldg(src + pos[i][j]);
                emit_store_col(v, (unsigned int *)e.dst[c], rbeg, nrow, pair_rows, e.vec, lane);
            }
        }
        if (e.rid_out[j]) {
            unsigned int v[EMIT_RPT];
#pragma unroll
            for (int i = 0; i < EMIT_RPT; i++) v[i] = __ldg(e.perm[j] + pos[i][j]);
            emit_store_col(v, e.rid_out[j], rbeg, nrow, pair_rows,
                           e.vec && ((uintptr_t)e.rid_out[j] & 31) == 0, lane);
        }
    }
}

template <int K>
cudaError_t launch_k(Ctx &c, const Emit4Spec &s, const uint32_t *B_dev, uint64_t row0, int64_t n) {
    const int64_t tiles = ceil_div(n, EMIT4_TILE);
    uint32_t *tile_first = nullptr;
    GJ_CUDA_TRY(dalloc(c, &tile_first, tiles + 1));
    // at most one block per row of the window
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, EMIT_DT), (int64_t)c.num_sms * 16));
    k_tile_first<<<(unsigned)grid, EMIT_DT, 0, c.stream>>>(s.A, B_dev, row0, n, tiles, tile_first); c.launches++;
    if (c.prof) cudaEventRecord(c.event(), c.stream);
    k_emit4<K><<<(unsigned)tiles, EMIT_DT, 0, c.stream>>>(s, tile_first, tiles, B_dev, row0, n); c.launches++;
    cudaError_t e = cudaGetLastError();
    dfree(c, tile_first);
    return e;
}

}  // namespace

cudaError_t launch_emit(Ctx &c, int k, const Emit4Spec &s, const uint32_t *B_dev, uint64_t row0,
                        int64_t n) {
    switch (k) {
        case 1: return launch_k<1>(c, s, B_dev, row0, n);
        case 2: return launch_k<2>(c, s, B_dev, row0, n);
        case 3: return launch_k<3>(c, s, B_dev, row0, n);
        case 4: return launch_k<4>(c, s, B_dev, row0, n);
        case 5: return launch_k<5>(c, s, B_dev, row0, n);
        case 6: return launch_k<6>(c, s, B_dev, row0, n);
        case 7: return launch_k<7>(c, s, B_dev, row0, n);
        case 8: return launch_k<8>(c, s, B_dev, row0, n);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gj
