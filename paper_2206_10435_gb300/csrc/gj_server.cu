// gj_server.cu -- native serving runtime: a stream of join queries over
// resident relations, continuously admitted into concurrent slots.
//
// A dispatcher thread releases the requests of a trace at their arrival
// times and plans each one (gj_query_create: host work only once the
// factors exist); admission is FIFO and takes the head request only while
// the estimated device memory of all admitted requests stays under the HBM
// budget.  Each slot is a host thread with its own CUDA stream: it gives
// the query that stream (gj_query_set_stream), summarises it (one
// synchronisation), then streams its result rows chunk by chunk (up to the
// server's row limit) through the slot's buffers, hashing every chunk on the
// device, so requests that arrive while others are on the GPU overlap with
// them as soon as a slot and memory are free.  Admission counts the bytes the
// context's memory pool has actually handed out plus the new request's
// estimate.  Times are taken on the host's steady clock from the request's
// arrival.
#include <math.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>

#include "gj_state.cuh"

namespace gj {

gj_status desummarize(QueryState &q, uint64_t row0, uint64_t nrows, void *const *out_cols,
                      uint32_t *const *rowid_cols, uint64_t *n_out);

namespace {

// Order-independent, position-dependent hash of a result chunk: the
// xor over rows and columns of a 64-bit mix of (column, row, value).
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

// every column of a chunk in one launch (blockIdx.y = column)
struct ChunkCols {
    int n;
    const void *col[64];
    int width[64];
};

__global__ void k_chunk_hash(ChunkCols cc, uint64_t row0, int64_t n, unsigned long long *h) {
    const int c = blockIdx.y;
    const void *col = cc.col[c];
    const int width = cc.width[c];
    uint64_t acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t v = width == 8 ? ((const uint64_t *)col)[i] : (uint64_t)((const uint32_t *)col)[i];
        acc ^= mix64(v ^ mix64(((uint64_t)c << 40) ^ (row0 + (uint64_t)i)));
    }
    for (int d = 16; d; d >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0 && acc) atomicXor(h, (unsigned long long)acc);
}

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct Pending {
    int idx;
    gj_query *q;
    uint64_t est;
};

struct ServerState {
    gj_ctx *ctx = nullptr;
    int n_slots = 0;
    uint64_t budget = 0, chunk = 0;
    uint64_t max_rows = 0;                       // rows streamed per request (0: all)
    // per slot: an execution context (stream, readback buffer, error word)
    // lent to the queries the slot runs, so a request allocates nothing
    std::vector<std::unique_ptr<Ctx>> exec;
    std::vector<cudaStream_t> streams;
    // each slot allocates from a memory pool of its own, so slots do not
    // contend for one pool's lock
    std::vector<cudaMemPool_t> pools;
    std::vector<std::vector<void *>> bufs;       // column buffers, chunk rows each
    std::vector<std::vector<int>> buf_width;
    std::vector<unsigned long long *> hash;
    std::vector<uint64_t *> hash_host;           // pinned
    // run state
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> pending;
    uint64_t used = 0, peak_used = 0;
    int in_flight = 0, peak_in_flight = 0;
    int remaining = 0;
    bool stop = false;
    gj_request_result *results = nullptr;
};

namespace {

// bytes the context's memory pool and the slots' pools have handed out and
// not taken back
uint64_t pool_bytes(ServerState &S) {
    uint64_t total = 0;
    bool any = false;
    auto add = [&](cudaMemPool_t pool) {
        if (!pool) return;
        size_t v = 0;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v) == cudaSuccess) {
            total += (uint64_t)v;
            any = true;
        } else {
            cudaGetLastError();
        }
    };
    add(S.ctx->s.c.pool);
    for (cudaMemPool_t p : S.pools) add(p);
    return any ? total : S.used;
}

void run_one(ServerState &S, int slot, Pending &p) {
    gj_request_result &r = S.results[p.idx];
    gj_query *q = p.q;
    r.slot = slot;
    Ctx &x = *S.exec[slot];
    q->s.exec = &x;
    gj_status st = GJ_OK;
    uint64_t total = 0;
    // the request's device memory comes from the slot's arena while it has
    // room: no allocator calls (which every slot's thread would otherwise
    // make by the dozen per request) and frees that cost nothing.  The
    // arena starts empty: the previous request's work was enqueued on this
    // same stream, before anything that reuses its memory.
    x.arena_used = 0;
    x.arena_on = x.arena != nullptr;
    if (st == GJ_OK) st = gj_summarize(q, &total);
    x.arena_on = false;   // the slot's long-lived buffers below come from the pool
    r.total = total;
    r.t_summary = now_s();
    if (st == GJ_OK && total > 0) {
        QueryState &qs = q->s;
        // output columns of this query: V keys (int32) then payloads
        std::vector<int> widths;
        for (size_t v = 0; v < qs.var_rel.size(); v++) widths.push_back(4);
        for (size_t p2 = 0; p2 < qs.col_rel.size(); p2++)
            widths.push_back(qs.r[qs.col_rel[p2]].R->pw[qs.col_pay[p2]]);
        std::vector<void *> &bufs = S.bufs[slot];
        std::vector<int> &bw = S.buf_width[slot];
        Ctx &c = qs.ctx();
        while (bufs.size() < widths.size()) { bufs.push_back(nullptr); bw.push_back(0); }
        for (size_t i = 0; i < widths.size() && st == GJ_OK; i++) {
            if (!bufs[i]) {   // 8-byte wide, so any column fits; kept for the slot's life
                if (dalloc_bytes(c, &bufs[i], (size_t)8 * S.chunk) != cudaSuccess) st = GJ_ERR_OOM;
                bw[i] = 8;
            }
        }
        // stream the result (up to the row limit) chunk by chunk; the hash
        // of every chunk accumulates on the device, and each chunk's
        // desummarisation waits for the previous one to be hashed.  A
        // chunk's temporaries come from the slot's arena past the summary's
        // arrays and are rewound after it (later chunks reuse them in
        // stream order).
        const uint64_t want = S.max_rows ? std::min<uint64_t>(S.max_rows, total) : total;
        if (st == GJ_OK) cudaMemsetAsync(S.hash[slot], 0, 8, c.stream);
        const size_t mark = c.arena_used;
        c.arena_on = c.arena != nullptr;
        uint64_t done = 0;
        while (st == GJ_OK && done < want) {
            uint64_t n = 0;
            c.arena_used = mark;
            st = desummarize(qs, done, std::min<uint64_t>(S.chunk, want - done), bufs.data(), nullptr, &n);
            if (st != GJ_OK || n == 0) break;
            ChunkCols cc{};
            cc.n = (int)widths.size();
            for (int i = 0; i < cc.n && i < 64; i++) { cc.col[i] = bufs[i]; cc.width[i] = widths[i]; }
            const int cols = std::min(cc.n, 64);
            const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)n, 256),
                                                                      std::max<int64_t>(1, c.num_sms * 4 / cols)));
            k_chunk_hash<<<dim3(gx, cols), 256, 0, c.stream>>>(cc, done, (int64_t)n, S.hash[slot]);
            if (done == 0) r.t_chunk = now_s();   // the first chunk is out (desummarise waited for it)
            done += n;
        }
        r.rows = done;
        if (st == GJ_OK) {
            cudaMemcpyAsync(S.hash_host[slot], S.hash[slot], 8, cudaMemcpyDeviceToHost, c.stream);
            if (cudaStreamSynchronize(c.stream) != cudaSuccess) { cudaGetLastError(); st = GJ_ERR_CUDA; }
            r.hash = S.hash_host[slot][0];
        }
    }
    x.arena_on = false;
    r.status = st;
    r.t_last = now_s();
    if (r.t_chunk == 0) r.t_chunk = r.t_last;
}

void worker(ServerState *S, int slot) {
    int dev = S->ctx->s.c.device;
    cudaSetDevice(dev);
    for (;;) {
        Pending p;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (!S->pending.empty()) {
                    Pending &h = S->pending.front();
                    // bytes the pool has handed out (resident factors, the
                    // summaries and buffers of the requests in flight) plus
                    // the new request's estimate
                    const uint64_t in_use = pool_bytes(*S) ;
                    if (in_use + h.est <= S->budget) break;
                    if (S->in_flight == 0) {
                        // nothing will free memory: it can never be admitted
                        Pending p = h;
                        S->pending.pop_front();
                        gj_request_result &r = S->results[p.idx];
                        r.status = GJ_ERR_OOM;
                        r.t_admit = r.t_summary = r.t_chunk = r.t_last = now_s();
                        gj_query_destroy(p.q);
                        S->remaining--;
                        S->cv.notify_all();
                        continue;
                    }
                }
                if (S->stop && S->pending.empty()) return;
                S->cv.wait(lk);
            }
            p = S->pending.front();
            S->pending.pop_front();
            S->used += p.est;
            S->peak_used = std::max(S->peak_used, pool_bytes(*S) + p.est);
            S->in_flight++;
            S->peak_in_flight = std::max(S->peak_in_flight, S->in_flight);
            S->results[p.idx].t_admit = now_s();
        }
        run_one(*S, slot, p);
        gj_query_destroy(p.q);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->used -= p.est;
            S->in_flight--;
            S->remaining--;
        }
        S->cv.notify_all();
    }
}

}  // namespace
}  // namespace gj

struct gj_server {
    gj::ServerState s;
};

using namespace gj;

extern "C" {

gj_status gj_server_create(gj_ctx *ctx, int32_t n_slots, uint64_t hbm_budget, uint64_t chunk_rows,
                           uint64_t max_rows, gj_server **out) {
    if (!ctx || !out || n_slots < 1 || n_slots > 256 || chunk_rows < 1 || chunk_rows > (1ull << 31))
        return GJ_ERR_INVALID;
    *out = nullptr;
    std::unique_ptr<gj_server> sv(new gj_server());
    ServerState &S = sv->s;
    S.ctx = ctx;
    S.n_slots = n_slots;
    S.budget = hbm_budget;
    S.chunk = chunk_rows;
    S.max_rows = max_rows;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->s.c.device);
    gj_status st = GJ_OK;
    for (int i = 0; i < n_slots && st == GJ_OK; i++) {
        cudaStream_t s = nullptr;
        unsigned long long *h = nullptr;
        uint64_t *hh = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc((void **)&h, 8) != cudaSuccess ||
            cudaMallocHost((void **)&hh, 8) != cudaSuccess) {
            cudaGetLastError();
            st = GJ_ERR_CUDA;
        }
        S.streams.push_back(s);
        S.hash.push_back(h);
        S.hash_host.push_back(hh);
        std::unique_ptr<Ctx> x(new Ctx());
        x->device = ctx->s.c.device;
        x->pool = ctx->s.c.pool;
        {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = ctx->s.c.device;
            cudaMemPool_t pool = nullptr;
            if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
                uint64_t keep = ~0ull;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
                x->pool = pool;
            } else {
                cudaGetLastError();   // the context's pool then
            }
            S.pools.push_back(pool);
        }
        x->num_sms = ctx->s.c.num_sms;
        x->emit_rpt = ctx->s.c.emit_rpt;
        x->tri_mode = ctx->s.c.tri_mode;
        x->down_combine = ctx->s.c.down_combine;
        x->stream = s;
        if (st == GJ_OK && (cudaMalloc((void **)&x->err, 16) != cudaSuccess ||
                            cudaMallocHost((void **)&x->pinned, 1 << 16) != cudaSuccess)) {
            cudaGetLastError();
            st = GJ_ERR_CUDA;
        }
        if (x->err) cudaMemset(x->err, 0, 16);
        // the slot's arena, from its pool (so that admission counts it)
        // (a request that needs more -- summary, and each result chunk's
        // temporaries -- continues in the slot's pool)
        const size_t arena = ctx->s.c.slot_arena;
        if (st == GJ_OK && arena > 0) {
            void *a = nullptr;
            cudaError_t e = x->pool ? cudaMallocFromPoolAsync(&a, arena, x->pool, s)
                                    : cudaMallocAsync(&a, arena, s);
            if (e == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess) {
                x->arena = (char *)a;
                x->arena_size = arena;
            } else {
                cudaGetLastError();   // no arena: the slot allocates from its pool
            }
        }
        S.exec.push_back(std::move(x));
    }
    S.bufs.assign(n_slots, {});
    S.buf_width.assign(n_slots, {});
    if (prev >= 0) cudaSetDevice(prev);
    if (st != GJ_OK) { gj_server_destroy(sv.release()); return st; }
    *out = sv.release();
    return GJ_OK;
}

gj_status gj_server_run(gj_server *sv, int32_t n_requests, const int32_t *rel_ids,
                        const int32_t *query_off, const double *arrival_offsets,
                        gj_request_result *results, gj_server_stats *stats) {
    if (!sv || n_requests < 0 || !rel_ids || !query_off || !arrival_offsets || !results)
        return GJ_ERR_INVALID;
    ServerState &S = sv->s;
    memset(results, 0, sizeof(gj_request_result) * (size_t)n_requests);
    S.results = results;
    S.pending.clear();
    S.used = S.peak_used = 0;
    S.in_flight = S.peak_in_flight = 0;
    S.remaining = n_requests;
    S.stop = false;
    std::vector<std::thread> threads;
    for (int i = 0; i < S.n_slots; i++) threads.emplace_back(worker, &S, i);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S.ctx->s.c.device);
    const double t0 = now_s();
    for (int i = 0; i < n_requests; i++) {
        const double due = t0 + arrival_offsets[i];
        double t = now_s();
        if (due > t) std::this_thread::sleep_for(std::chrono::duration<double>(due - t));
        gj_request_result &r = results[i];
        r.t_arrival = now_s();
        gj_query *q = nullptr;
        gj_status st = gj_query_create(S.ctx, rel_ids + query_off[i], query_off[i + 1] - query_off[i], &q);
        if (st != GJ_OK) {
            r.status = st;
            r.t_summary = r.t_chunk = r.t_last = now_s();
            std::lock_guard<std::mutex> lk(S.mu);
            S.remaining--;
            continue;
        }
        // device memory of the summary (about 80 bytes per group) and of the
        // first chunk's window expansion
        uint64_t groups = 0;
        for (auto &t : q->s.r) groups += (uint64_t)t.F->G;
        const uint64_t est = 80 * groups + 2 * S.chunk * (16 + 4 * (uint64_t)q->s.k) + (1u << 20);
        r.est_bytes = est;
        if (est > S.budget) {
            r.status = GJ_ERR_OOM;   // can never be admitted
            r.t_summary = r.t_chunk = r.t_last = now_s();
            gj_query_destroy(q);
            std::lock_guard<std::mutex> lk(S.mu);
            S.remaining--;
            continue;
        }
        {
            std::lock_guard<std::mutex> lk(S.mu);
            S.pending.push_back(Pending{i, q, est});
        }
        S.cv.notify_all();
    }
    {
        std::unique_lock<std::mutex> lk(S.mu);
        S.cv.wait(lk, [&] { return S.remaining == 0; });
        S.stop = true;
    }
    S.cv.notify_all();
    for (auto &th : threads) th.join();
    if (prev >= 0) cudaSetDevice(prev);
    if (stats) {
        stats->peak_in_flight = S.peak_in_flight;
        stats->peak_admitted_bytes = S.peak_used;
        stats->wall_s = now_s() - t0;
    }
    S.results = nullptr;
    return GJ_OK;
}

void gj_server_destroy(gj_server *sv) {
    if (!sv) return;
    ServerState &S = sv->s;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S.ctx->s.c.device);
    for (int i = 0; i < (int)S.streams.size(); i++) {
        if (S.streams[i]) cudaStreamSynchronize(S.streams[i]);
        for (void *b : S.bufs[i]) if (b) cudaFreeAsync(b, S.streams[i]);
        if (S.streams[i]) cudaStreamSynchronize(S.streams[i]);
        if (S.hash[i]) cudaFree(S.hash[i]);
        if (S.hash_host[i]) cudaFreeHost(S.hash_host[i]);
        if (i < (int)S.exec.size() && S.exec[i]) {
            if (S.exec[i]->arena) cudaFreeAsync(S.exec[i]->arena, S.streams[i]);
            if (S.exec[i]->err) cudaFree(S.exec[i]->err);
            if (S.exec[i]->pinned) cudaFreeHost(S.exec[i]->pinned);
        }
        if (S.streams[i]) cudaStreamDestroy(S.streams[i]);
        if (i < (int)S.pools.size() && S.pools[i]) cudaMemPoolDestroy(S.pools[i]);
    }
    if (prev >= 0) cudaSetDevice(prev);
    delete sv;
}

}  // extern "C"
