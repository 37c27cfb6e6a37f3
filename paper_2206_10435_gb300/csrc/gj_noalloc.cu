// gj_noalloc.cu -- factor construction for callers that cannot allocate.
//
// Some callers cannot allocate device memory: a database engine or a
// serving process that hands all device memory to its own pool (where a
// cudaMalloc would fail, or break the pool's accounting), or code on a
// latency-critical path where cudaMalloc/cudaFree would synchronise the
// device.  gj_factor_build_noalloc gives them the frequency table of one
// relation with every scratch buffer carved out of one file-scope device
// array of fixed size, g_scratch below.  The caller still passes the
// inputs and the outputs.
//
// g_scratch exists once per device that loads the library and stays
// allocated until the process exits.  In host code its name is only a
// host-side stand-in: its device address is looked up with
// cudaGetSymbolAddress (once per device, with that device current) and that
// address is what the kernels receive.  Every call shares the array, so two
// calls whose work overlaps on the GPU race; everything that must start at
// zero (counters, lookback state, the error word) is cleared by each call.
#include <mutex>

#include "gj_state.cuh"

namespace gj {

cudaError_t factor_build_in(Ctx &c, const int32_t *const *cols, int nk, int64_t n,
                            const std::vector<int> &order, uint32_t *perm, uint32_t *gstart,
                            int32_t *gkey, int64_t *G_out, const FactorScratch &s);
size_t scan_u32_state_bytes(int64_t n);

namespace {

constexpr int64_t NA_ROWS = GJ_NOALLOC_MAX_ROWS;
// onesweep tiles of the sort (one status word per tile and digit value)
constexpr int64_t NA_TILES = (NA_ROWS + RADIX_SORT_TILE - 1) / RADIX_SORT_TILE;
constexpr size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr size_t OFF_ERR = 0;
constexpr size_t OFF_KEYS = 256;
constexpr size_t OFF_K2 = OFF_KEYS + a256(8 * NA_ROWS);
constexpr size_t OFF_V2 = OFF_K2 + a256(8 * NA_ROWS);
constexpr size_t OFF_HIST = OFF_V2 + a256(4 * NA_ROWS);
constexpr size_t HIST_WORDS = RADIX_SORT_MAX_PASSES * RADIX_SORT_BINS + RADIX_SORT_MAX_PASSES;
constexpr size_t OFF_STATUS = OFF_HIST + a256(4 * HIST_WORDS);
constexpr size_t OFF_HEAD = OFF_STATUS + a256(8 * RADIX_SORT_BINS * NA_TILES);
constexpr size_t OFF_GID = OFF_HEAD + a256(NA_ROWS);
constexpr size_t OFF_GCOUNT = OFF_GID + a256(4 * NA_ROWS);
constexpr size_t OFF_MM = OFF_GCOUNT + 256;
constexpr size_t OFF_SCAN = OFF_MM + 256;
constexpr size_t SCAN_BYTES = scan_u32_state_bytes_for(NA_ROWS);
constexpr size_t SCRATCH_BYTES = OFF_SCAN + a256(SCAN_BYTES);
static_assert(2 * 4 * MAX_KEYS <= 256, "the key ranges fit their 256-byte slot");
static_assert(SCRATCH_BYTES < (8u << 20), "the fixed scratch stays under 8 MB");

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

std::mutex g_mu;
unsigned char *g_addr[256] = {};   // device address of g_scratch, per device

}  // namespace
}  // namespace gj

using namespace gj;

extern "C" gj_status gj_factor_build_noalloc(int32_t device, void *cuda_stream, int64_t n_rows,
                                             int32_t n_keys, const int32_t *const *key_cols,
                                             const int32_t *col_order, uint32_t *perm_dev,
                                             uint32_t *gstart_dev, int32_t *gkey_dev,
                                             int64_t *n_groups) {
    if (!n_groups) return GJ_ERR_INVALID;
    *n_groups = 0;
    if (n_rows < 0 || n_rows > NA_ROWS) return GJ_ERR_INVALID;   // beyond the fixed scratch
    if (n_keys < 1 || n_keys > MAX_KEYS || !key_cols) return GJ_ERR_INVALID;
    if (device < 0 || device >= 256) return GJ_ERR_INVALID;
    if (!gstart_dev || (n_rows > 0 && (!perm_dev || !gkey_dev))) return GJ_ERR_INVALID;
    std::vector<int> order(n_keys);
    {
        std::vector<int> seen(n_keys, 0);
        for (int i = 0; i < n_keys; i++) {
            int c = col_order ? col_order[i] : i;
            if (c < 0 || c >= n_keys || seen[c]) return GJ_ERR_INVALID;
            seen[c] = 1;
            order[i] = c;
        }
        for (int i = 0; i < n_keys; i++)
            if (n_rows > 0 && !key_cols[i]) return GJ_ERR_INVALID;
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); return GJ_ERR_CUDA; }
    if (prev != device && cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return GJ_ERR_CUDA; }
    gj_status st = GJ_OK;
    unsigned char *base = nullptr;
    {
        // first call on this device: look up the array's device address
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p) { cudaGetLastError(); st = GJ_ERR_CUDA; }
            else g_addr[device] = (unsigned char *)p;
        }
        base = g_addr[device];
    }
    if (st == GJ_OK) {
        Ctx c;
        c.device = device;
        c.stream = (cudaStream_t)cuda_stream;
        c.err = (uint32_t *)(base + OFF_ERR);
        cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, device);
        FactorScratch s{};
        s.keys = (uint64_t *)(base + OFF_KEYS);
        s.k2 = (uint64_t *)(base + OFF_K2);
        s.v2 = (uint32_t *)(base + OFF_V2);
        s.hist = (uint32_t *)(base + OFF_HIST);
        s.status = (unsigned long long *)(base + OFF_STATUS);
        s.status_tiles = NA_TILES;
        s.head = base + OFF_HEAD;
        s.gid = (uint32_t *)(base + OFF_GID);
        s.gcount = (uint32_t *)(base + OFF_GCOUNT);
        s.mm = (int32_t *)(base + OFF_MM);
        s.scan_state = base + OFF_SCAN;
        s.scan_state_bytes = SCAN_BYTES;
        cudaError_t e = cudaMemsetAsync(c.err, 0, 4, c.stream);
        int64_t G = 0;
        if (e == cudaSuccess)
            e = factor_build_in(c, key_cols, n_keys, n_rows, order, perm_dev, gstart_dev, gkey_dev,
                                &G, s);
        uint32_t err = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&err, c.err, 4, cudaMemcpyDeviceToHost, c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        if (e != cudaSuccess) { cudaGetLastError(); st = GJ_ERR_CUDA; }
        else if (err & ERRF_TIMEOUT) st = GJ_ERR_TIMEOUT;
        else if (err) st = GJ_ERR_CUDA;
        else *n_groups = G;
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return st;
}
