// gj_emit.cuh -- the desummarise emit kernel's launch description.
#pragma once

#include "gj_state.cuh"

namespace gj {

constexpr int EMIT_DT = 256;
constexpr int EMIT_MAXR = MAX_REL;
constexpr int EMIT_MAXV = 32;
constexpr int EMIT_MAXP = 32;
constexpr int MAXC = EMIT_MAXV + EMIT_MAXP;

struct Emit4Spec {
    const uint32_t *gstart[EMIT_MAXR];    // by query position
    const uint32_t *perm[EMIT_MAXR];
    uint32_t *rid_out[EMIT_MAXR];
    const uint32_t *grp[EMIT_MAXR];       // frontier groups, by query position
    int col_off[EMIT_MAXR + 1];           // output columns of relation j: [col_off[j], col_off[j+1])
    const void *src[MAXC];
    void *dst[MAXC];
    uint8_t kind[MAXC];              // 0 key (int32, by group), 1 payload int32, 2 payload int64
    const uint64_t *A;
    uint32_t *err;
    int vec;                         // every destination is 16-byte aligned
};


// Emits result rows [row0, row0 + n) from the block list A with the emit
// kernel for K = k relations (k <= 8).  B_dev: number of blocks, in device
// memory.  tile_first: the block holding the first row of every tile of
// EMIT_DT * c.emit_rpt rows, or NULL to have it computed here (a binary
// search of the block offsets per tile).
cudaError_t launch_emit(Ctx &c, int k, const Emit4Spec &s, const uint32_t *B_dev, uint64_t row0,
                        int64_t n, const uint32_t *tile_first = nullptr);

}  // namespace gj
