// emit_pattern.cu -- what bandwidth the desummarise emit's memory pattern
// allows on this GPU, without any of its index arithmetic.
//
// The emit writes a result window column by column (6 int32 key columns and
// 5 int64 payload columns for the 5-chain: 64 B per row) and, per row,
// gathers one payload per relation.  Inside a block (one group per
// relation) the payloads of relations 1..4 stay the same for many rows and
// the last relation's run through a contiguous range.  This program writes
// 2^28 such rows with the emit's thread layout (2048 rows per CTA, lanes 32
// rows apart) and times, with CUDA events, best of 5:
//   * a plain fill of one 16 GB array (the write ceiling);
//   * the 11 columns with no loads;
//   * the 11 columns with the gathers of blocks of 8, 64 and 256 rows, the
//     gathered arrays either 5 x 64 MB (larger than L2, like the factors of
//     the 5-chain) or 5 x 8 MB (L2-resident).
// Standalone (no library): nvcc -gencode arch=compute_103a,code=sm_103a -O3
//   -o emit_pattern emit_pattern.cu && ./emit_pattern
#include <cstdint>
#include <cstdio>
#include <vector>

#include <cuda_runtime.h>

#define CK(x)                                                                        \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess) {                                                     \
            printf("CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__);  \
            return 1;                                                                \
        }                                                                            \
    } while (0)

__global__ void fill1(uint64_t *p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        __stcs(p + i, (uint64_t)i);
}

struct Cols {
    uint32_t *k[6];
    uint64_t *p[5];
    const uint64_t *src[5];
};

// RUN == 0: no loads; RUN > 0: blocks of RUN rows, gathered index masked
// into the source arrays (mask + 1 elements each)
template <int RUN>
__global__ void __launch_bounds__(256) fill_cols(Cols c, int64_t n, uint32_t mask) {
    const int64_t r0 = (int64_t)blockIdx.x * 2048;
    int rel = (threadIdx.x >> 5) * 256 + (threadIdx.x & 31);
#pragma unroll 1
    for (int i = 0; i < 8; i++, rel += 32) {
        const int64_t R = r0 + rel;
        if (R >= n) break;
#pragma unroll
        for (int s = 0; s < 6; s++) __stcs(c.k[s] + R, (uint32_t)R + s);
#pragma unroll
        for (int j = 0; j < 5; j++) {
            uint64_t v = (uint64_t)R * (j + 1);
            if (RUN > 0) {
                const uint32_t blk = (uint32_t)(R / (RUN > 0 ? RUN : 1));
                const uint32_t b0 = (blk * 2654435761u + j * 40503u) & mask;
                const uint32_t at = j == 4 ? ((b0 + (uint32_t)(R % (RUN > 0 ? RUN : 1))) & mask) : b0;
                v = __ldg(c.src[j] + at);
            }
            __stcs(c.p[j] + R, v);
        }
    }
}

int main() {
    const int64_t n = 1ll << 28;        // rows
    const int64_t srcn = 1ll << 23;     // elements per gathered array (64 MB)
    Cols c;
    std::vector<void *> all;
    for (int s = 0; s < 6; s++) { CK(cudaMalloc(&c.k[s], n * 4)); all.push_back(c.k[s]); }
    for (int j = 0; j < 5; j++) { CK(cudaMalloc(&c.p[j], n * 8)); all.push_back(c.p[j]); }
    for (int j = 0; j < 5; j++) {
        uint64_t *s;
        CK(cudaMalloc(&s, srcn * 8));
        CK(cudaMemset(s, 1, srcn * 8));
        c.src[j] = s;
        all.push_back(s);
    }
    const int64_t nb = 1ll << 31;
    uint64_t *big;
    CK(cudaMalloc(&big, nb * 8));
    all.push_back(big);
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    auto run = [&](const char *name, double bytes, auto launch) {
        for (int w = 0; w < 3; w++) launch();
        cudaDeviceSynchronize();
        float best = 1e30f;
        for (int r = 0; r < 5; r++) {
            cudaEventRecord(a);
            launch();
            cudaEventRecord(b);
            cudaEventSynchronize(b);
            float ms;
            cudaEventElapsedTime(&ms, a, b);
            if (ms < best) best = ms;
        }
        printf("%-34s %8.3f ms %8.1f GB/s\n", name, best, bytes / best / 1e6);
    };
    const unsigned tiles = (unsigned)(n / 2048);
    const uint32_t big_mask = (uint32_t)(srcn - 1), l2_mask = (1u << 20) - 1;
    run("fill, one 16 GB array", nb * 8.0, [&] { fill1<<<152 * 8, 1024>>>(big, nb); });
    run("11 columns, no loads", n * 64.0, [&] { fill_cols<0><<<tiles, 256>>>(c, n, big_mask); });
    run("blocks of 8, 5 x 64 MB gathered", n * 64.0, [&] { fill_cols<8><<<tiles, 256>>>(c, n, big_mask); });
    run("blocks of 8, 5 x 8 MB gathered", n * 64.0, [&] { fill_cols<8><<<tiles, 256>>>(c, n, l2_mask); });
    run("blocks of 64, 5 x 64 MB gathered", n * 64.0, [&] { fill_cols<64><<<tiles, 256>>>(c, n, big_mask); });
    run("blocks of 256, 5 x 64 MB gathered", n * 64.0, [&] { fill_cols<256><<<tiles, 256>>>(c, n, big_mask); });
    run("blocks of 256, 5 x 8 MB gathered", n * 64.0, [&] { fill_cols<256><<<tiles, 256>>>(c, n, l2_mask); });
    CK(cudaGetLastError());
    for (void *p : all) cudaFree(p);
    return 0;
}
