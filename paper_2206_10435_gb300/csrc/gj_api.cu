// gj_api.cu -- the C ABI of include/gj.h: contexts, relations, the join-tree
// planner and the entry points of the three steps.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <set>

#include "gj_state.cuh"

namespace gj {

cudaError_t relation_minmax(Ctx &c, Relation &R);
cudaError_t factor_build(Ctx &c, Relation &R, const std::vector<int> &order, Factor &F);
cudaError_t factor_build_many(Ctx &c, const std::vector<Relation *> &R, const std::vector<Factor *> &F);
void factor_free(Ctx &c, Factor &F);
void query_free_summary(Ctx &c, QueryState &q);
gj_status summarize(QueryState &q, uint64_t *total_out);
bool plan_cyclic(QueryState &q);
gj_status desummarize(QueryState &q, uint64_t row0, uint64_t nrows, void *const *out_cols,
                      uint32_t *const *rowid_cols, uint64_t *n_out);
gj_status level_runs(QueryState &q, int level, uint64_t row0, uint64_t nrows, int32_t *val,
                     uint64_t *freq, uint64_t *off, uint64_t cap, uint64_t *n_out);

static thread_local char g_last_error[256] = "";

void note_cuda_error(cudaError_t e, const char *file, int line) {
    const char *base = strrchr(file, '/');
    snprintf(g_last_error, sizeof(g_last_error), "%s (%s) at %s:%d", cudaGetErrorName(e),
             cudaGetErrorString(e), base ? base + 1 : file, line);
}

gj_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return GJ_OK;
    cudaGetLastError();   // clear sticky-free errors
    return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
}

// Reads and clears the device error word (synchronises the stream).
gj_status check_device_error(Ctx &c) {
    uint32_t *h = (uint32_t *)c.pinned;
    if (cudaMemcpyAsync(h, c.err, 4, cudaMemcpyDeviceToHost, c.stream) != cudaSuccess)
        return GJ_ERR_CUDA;
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return GJ_ERR_CUDA;
    uint32_t e = h[0];
    if (e) cudaMemsetAsync(c.err, 0, 4, c.stream);
    if (e & ERRF_TIMEOUT) return GJ_ERR_TIMEOUT;
    if (e) return GJ_ERR_CUDA;
    return GJ_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        // always: in a thread that has not used CUDA yet this also makes the
        // device's primary context current (cudaGetDevice alone reports
        // device 0 without doing so, and pointer queries then fail)
        cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

Factor *get_factor(CtxState &cs, Relation &R, const std::vector<int> &order, gj_status *st) {
    auto it = R.factors.find(order);
    if (it != R.factors.end()) { *st = GJ_OK; return it->second.get(); }
    std::unique_ptr<Factor> F(new Factor());
    cudaError_t e = factor_build(cs.c, R, order, *F);
    if (e != cudaSuccess) {
        factor_free(cs.c, *F);
        *st = from_cuda(e);
        return nullptr;
    }
    *st = check_device_error(cs.c);
    if (*st != GJ_OK) { factor_free(cs.c, *F); return nullptr; }
    Factor *p = F.get();
    R.factors[order] = std::move(F);
    return p;
}

bool valid_order(const Relation &R, const int32_t *col_order, std::vector<int> &order) {
    order.resize(R.nk);
    std::vector<int> seen(R.nk, 0);
    for (int i = 0; i < R.nk; i++) {
        int c = col_order ? col_order[i] : i;
        if (c < 0 || c >= R.nk || seen[c]) return false;
        seen[c] = 1;
        order[i] = c;
    }
    return true;
}

}  // namespace gj

using namespace gj;

extern "C" {

const char *gj_status_str(gj_status s) {
    switch (s) {
        case GJ_OK: return "ok";
        case GJ_ERR_INVALID: return "invalid argument";
        case GJ_ERR_NOT_ACYCLIC: return "relation order does not give a join tree";
        case GJ_ERR_OOM: return "device out of memory";
        case GJ_ERR_OVERFLOW: return "join size reaches 2^64 - 1";
        case GJ_ERR_CUDA: return "CUDA error";
        case GJ_ERR_TIMEOUT: return "device wait timed out";
        case GJ_ERR_STATE: return "call out of order";
        case GJ_ERR_CAPACITY: return "output buffer too small";
    }
    return "unknown status";
}

int32_t gj_version(void) { return 1; }

const char *gj_last_error(void) { return gj::g_last_error; }

gj_status gj_create(gj_ctx **out, int32_t device, void *cuda_stream) {
    if (!out) return GJ_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GJ_ERR_CUDA;
    }
    DeviceGuard g(device);
    gj_ctx *x = new gj_ctx();
    Ctx &c = x->s.c;
    c.device = device;
    c.stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc((void **)&c.err, 16) != cudaSuccess ||
        cudaMallocHost((void **)&c.pinned, 1 << 16) != cudaSuccess) {
        cudaGetLastError();
        if (c.err) cudaFree(c.err);
        delete x;
        return GJ_ERR_OOM;
    }
    cudaMemset(c.err, 0, 16);
    {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        if (cudaMemPoolCreate(&c.pool, &props) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(c.pool, cudaMemPoolAttrReleaseThreshold, &keep);
        } else {
            cudaGetLastError();
            c.pool = nullptr;   // fall back to the device's default pool
        }
    }
    cudaDeviceSynchronize();
    *out = x;
    return GJ_OK;
}

gj_status gj_profile(gj_ctx *ctx, int32_t enable, gj_profile_t *out) {
    if (!ctx) return GJ_ERR_INVALID;
    DeviceGuard g(ctx->s.c.device);
    Ctx &c = ctx->s.c;
    if (out) {
        if (cudaStreamSynchronize(c.stream) != cudaSuccess) return GJ_ERR_CUDA;
        double ms = 0;
        for (size_t i = 0; i + 1 < c.ev_used.size(); i += 2) {
            float t = 0;
            if (cudaEventElapsedTime(&t, c.ev_used[i], c.ev_used[i + 1]) == cudaSuccess) ms += t;
        }
        double xms = 0;
        for (size_t i = 0; i + 1 < c.xev_used.size(); i += 2) {
            float t = 0;
            if (cudaEventElapsedTime(&t, c.xev_used[i], c.xev_used[i + 1]) == cudaSuccess) xms += t;
        }
        c.ev_free.insert(c.ev_free.end(), c.ev_used.begin(), c.ev_used.end());
        c.ev_free.insert(c.ev_free.end(), c.xev_used.begin(), c.xev_used.end());
        c.ev_used.clear();
        c.xev_used.clear();
        out->expand_ms = xms;
        out->launches = c.launches;
        out->emit_launches = c.emit_launches;
        out->emit_ms = ms;
        out->emit_rows = c.emit_rows;
        out->emit_bytes = c.emit_bytes;
        c.launches = c.emit_launches = c.emit_rows = c.emit_bytes = 0;
    }
    c.prof = enable != 0;
    return GJ_OK;
}

gj_status gj_set_option(gj_ctx *ctx, int32_t option, int64_t value) {
    if (!ctx) return GJ_ERR_INVALID;
    if (option == GJ_OPT_EMIT_ROWS_PER_THREAD) {
        if (value != 2 && value != 4 && value != 8) return GJ_ERR_INVALID;
        ctx->s.c.emit_rpt = (int)value;
        return GJ_OK;
    }
    if (option == GJ_OPT_TRIANGLE_INTERSECT) {
        if (value < 0 || value > 2) return GJ_ERR_INVALID;
        ctx->s.c.tri_mode = (int)value;
        return GJ_OK;
    }
    if (option == GJ_OPT_DOWN_COMBINE) {
        if (value < 0 || value > 2) return GJ_ERR_INVALID;
        ctx->s.c.down_combine = (int)value;
        return GJ_OK;
    }
    if (option == GJ_OPT_SLOT_ARENA) {
        if (value < 0 || value > (1ll << 40)) return GJ_ERR_INVALID;
        ctx->s.c.slot_arena = (size_t)value;
        return GJ_OK;
    }
    if (option == GJ_OPT_SPIN_LIMIT) {
        if (value < 0 || value > (int64_t)SPIN_LIMIT) return GJ_ERR_INVALID;
        ctx->s.c.spin_limit = value == 0 ? SPIN_LIMIT : (uint32_t)value;
        return GJ_OK;
    }
    if (option == GJ_OPT_TEST_STALL) {
        if (value < 0 || value > 1) return GJ_ERR_INVALID;
        ctx->s.c.test_stall = value != 0;
        return GJ_OK;
    }
    if (option == GJ_OPT_FAIL_ALLOC_AT) {
        if (value < 0) return GJ_ERR_INVALID;
        ctx->s.c.fail_alloc_at = value;
        ctx->s.c.allocs = 0;
        return GJ_OK;
    }
    return GJ_ERR_INVALID;
}

gj_status gj_pool_usage(gj_ctx *ctx, uint64_t *used_bytes, int64_t *allocations) {
    if (!ctx) return GJ_ERR_INVALID;
    DeviceGuard g(ctx->s.c.device);
    Ctx &c = ctx->s.c;
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) { cudaGetLastError(); return GJ_ERR_CUDA; }
    if (used_bytes) {
        *used_bytes = 0;
        if (c.pool) {
            size_t v = 0;   // the attribute is a 64-bit value
            if (cudaMemPoolGetAttribute(c.pool, cudaMemPoolAttrUsedMemCurrent, &v) != cudaSuccess) {
                cudaGetLastError();
                return GJ_ERR_CUDA;
            }
            *used_bytes = (uint64_t)v;
        }
    }
    if (allocations) *allocations = c.allocs;
    return GJ_OK;
}

gj_status gj_set_stream(gj_ctx *ctx, void *cuda_stream) {
    if (!ctx) return GJ_ERR_INVALID;
    DeviceGuard g(ctx->s.c.device);
    cudaStreamSynchronize(ctx->s.c.stream);
    ctx->s.c.stream = (cudaStream_t)cuda_stream;
    return GJ_OK;
}

static void relation_free(Ctx &c, Relation &R) {
    for (auto &kv : R.factors) factor_free(c, *kv.second);
    R.factors.clear();
    for (void *&p : R.owned) dfree(c, p);
    R.owned.clear();
}

void gj_destroy(gj_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->s.c.device);
    Ctx &c = ctx->s.c;
    for (auto &kv : ctx->s.rels) relation_free(c, *kv.second);
    ctx->s.rels.clear();
    cudaStreamSynchronize(c.stream);
    if (c.pool) cudaMemPoolDestroy(c.pool);
    for (cudaEvent_t e : c.ev_free) cudaEventDestroy(e);
    for (cudaEvent_t e : c.ev_used) cudaEventDestroy(e);
    for (cudaEvent_t e : c.xev_used) cudaEventDestroy(e);
    cudaFree(c.err);
    cudaFreeHost(c.pinned);
    delete ctx;
}

gj_status gj_load_relation(gj_ctx *ctx, const gj_relation_desc *d, int32_t *rel_id) {
    if (!ctx) return GJ_ERR_INVALID;
    std::lock_guard<std::recursive_mutex> lock(ctx->s.mu);
    if (!ctx || !d || !rel_id) return GJ_ERR_INVALID;
    if (d->n_rows < 0 || d->n_rows > 0x7fffffffLL) return GJ_ERR_INVALID;
    if (d->n_keys < 1 || d->n_keys > MAX_KEYS) return GJ_ERR_INVALID;
    if (d->n_payloads < 0 || d->n_payloads > MAX_PAYLOADS) return GJ_ERR_INVALID;
    if (!d->key_attr || !d->key_cols) return GJ_ERR_INVALID;
    if (d->n_payloads && (!d->payload_width || !d->payload_cols)) return GJ_ERR_INVALID;
    std::set<int32_t> attrs;
    for (int i = 0; i < d->n_keys; i++) {
        if (!attrs.insert(d->key_attr[i]).second) return GJ_ERR_INVALID;
        if (d->n_rows > 0 && !d->key_cols[i]) return GJ_ERR_INVALID;
    }
    for (int i = 0; i < d->n_payloads; i++) {
        if (d->payload_width[i] != 4 && d->payload_width[i] != 8) return GJ_ERR_INVALID;
        if (d->n_rows > 0 && !d->payload_cols[i]) return GJ_ERR_INVALID;
    }
    DeviceGuard g(ctx->s.c.device);
    Ctx &c = ctx->s.c;
    std::unique_ptr<Relation> R(new Relation());
    R->n = d->n_rows;
    R->nk = d->n_keys;
    R->np = d->n_payloads;
    const bool copy = (d->flags & (GJ_REL_COPY | GJ_REL_HOST)) != 0;
    for (int i = 0; i < d->n_keys; i++) {
        R->attr.push_back(d->key_attr[i]);
        const int32_t *p = d->key_cols[i];
        if (copy && R->n > 0) {
            void *q = nullptr;
            if (dalloc_bytes(c, &q, 4 * R->n) != cudaSuccess) { relation_free(c, *R); return GJ_ERR_OOM; }
            R->owned.push_back(q);
            if (cudaMemcpyAsync(q, p, 4 * R->n, cudaMemcpyDefault, c.stream) != cudaSuccess) {
                relation_free(c, *R);
                return GJ_ERR_CUDA;
            }
            p = (const int32_t *)q;
        }
        R->key.push_back(p);
    }
    for (int i = 0; i < d->n_payloads; i++) {
        R->pw.push_back(d->payload_width[i]);
        const void *p = d->payload_cols[i];
        size_t bytes = (size_t)d->payload_width[i] * R->n;
        if (copy && R->n > 0) {
            void *q = nullptr;
            if (dalloc_bytes(c, &q, bytes) != cudaSuccess) { relation_free(c, *R); return GJ_ERR_OOM; }
            R->owned.push_back(q);
            if (cudaMemcpyAsync(q, p, bytes, cudaMemcpyDefault, c.stream) != cudaSuccess) {
                relation_free(c, *R);
                return GJ_ERR_CUDA;
            }
            p = q;
        }
        R->pay.push_back(p);
    }
    int32_t id = ctx->s.next_id++;
    ctx->s.rels[id] = std::move(R);
    *rel_id = id;
    return GJ_OK;
}

gj_status gj_release_relation(gj_ctx *ctx, int32_t rel_id) {
    if (!ctx) return GJ_ERR_INVALID;
    std::lock_guard<std::recursive_mutex> lock(ctx->s.mu);
    if (!ctx) return GJ_ERR_INVALID;
    auto it = ctx->s.rels.find(rel_id);
    if (it == ctx->s.rels.end()) return GJ_ERR_INVALID;
    DeviceGuard g(ctx->s.c.device);
    relation_free(ctx->s.c, *it->second);
    ctx->s.rels.erase(it);
    return GJ_OK;
}

gj_status gj_build_factors(gj_ctx *ctx, int32_t rel_id, const int32_t *col_order) {
    if (!ctx) return GJ_ERR_INVALID;
    std::lock_guard<std::recursive_mutex> lock(ctx->s.mu);
    if (!ctx) return GJ_ERR_INVALID;
    auto it = ctx->s.rels.find(rel_id);
    if (it == ctx->s.rels.end()) return GJ_ERR_INVALID;
    std::vector<int> order;
    if (!valid_order(*it->second, col_order, order)) return GJ_ERR_INVALID;
    DeviceGuard g(ctx->s.c.device);
    gj_status st;
    get_factor(ctx->s, *it->second, order, &st);
    return st;
}

gj_status gj_factor_export(gj_ctx *ctx, int32_t rel_id, const int32_t *col_order,
                           int64_t *n_groups, uint32_t *perm_dev, uint32_t *gstart_dev,
                           int32_t *gkey_dev) {
    if (!ctx) return GJ_ERR_INVALID;
    std::lock_guard<std::recursive_mutex> lock(ctx->s.mu);
    if (!ctx || !n_groups) return GJ_ERR_INVALID;
    auto it = ctx->s.rels.find(rel_id);
    if (it == ctx->s.rels.end()) return GJ_ERR_INVALID;
    Relation &R = *it->second;
    std::vector<int> order;
    if (!valid_order(R, col_order, order)) return GJ_ERR_INVALID;
    DeviceGuard g(ctx->s.c.device);
    gj_status st;
    Factor *F = get_factor(ctx->s, R, order, &st);
    if (!F) return st;
    Ctx &c = ctx->s.c;
    *n_groups = F->G;
    if (perm_dev && R.n)
        if (cudaMemcpyAsync(perm_dev, F->perm, 4 * R.n, cudaMemcpyDeviceToDevice, c.stream)) return GJ_ERR_CUDA;
    if (gstart_dev)
        if (cudaMemcpyAsync(gstart_dev, F->gstart, 4 * (F->G + 1), cudaMemcpyDeviceToDevice, c.stream)) return GJ_ERR_CUDA;
    if (gkey_dev && F->G)
        if (cudaMemcpyAsync(gkey_dev, F->gkey, 4 * R.nk * F->G, cudaMemcpyDeviceToDevice, c.stream)) return GJ_ERR_CUDA;
    return from_cuda(cudaStreamSynchronize(c.stream));
}

}  // extern "C"

namespace {

// The factors of the query's relations (factor order: separator columns,
// then the relation's own); the missing ones are built together, sharing
// their host synchronisations.
gj_status get_factors(CtxState &cs, std::vector<QRel> &ts) {
    std::vector<std::vector<int>> orders(ts.size());
    std::vector<Relation *> R;
    std::vector<Factor *> F;
    std::vector<std::unique_ptr<Factor>> made;
    for (size_t i = 0; i < ts.size(); i++) {
        orders[i] = ts[i].sep_cols;
        orders[i].insert(orders[i].end(), ts[i].new_cols.begin(), ts[i].new_cols.end());
        if (ts[i].R->factors.count(orders[i])) continue;
        bool dup = false;
        for (size_t k = 0; k < F.size() && !dup; k++) dup = R[k] == ts[i].R && F[k]->order == orders[i];
        if (dup) continue;
        made.emplace_back(new Factor());
        made.back()->order = orders[i];
        R.push_back(ts[i].R);
        F.push_back(made.back().get());
    }
    if (!F.empty()) {
        cudaError_t e = factor_build_many(cs.c, R, F);
        gj_status st = e == cudaSuccess ? check_device_error(cs.c) : from_cuda(e);
        if (st != GJ_OK) {
            for (auto &f : made) factor_free(cs.c, *f);
            return st;
        }
        for (size_t k = 0; k < made.size(); k++) R[k]->factors[F[k]->order] = std::move(made[k]);
    }
    for (size_t i = 0; i < ts.size(); i++) ts[i].F = ts[i].R->factors[orders[i]].get();
    return GJ_OK;
}

// The cyclic 3-way join (gj_cycle.cu): three relations of two distinct key
// attributes each, every pair sharing exactly one, the three shared
// attributes distinct (R0(A,B), R1(B,C), R2(C,A) up to column order).  Fills
// the plan: V = R0's columns in declared order, then R1's attribute C;
// factor orders R0 declared, R1 (B, C), R2 (A, C); payloads as usual.
bool plan_triangle(CtxState &cs, const int32_t *rel_ids, QueryState &q) {
    Relation *R[3];
    for (int j = 0; j < 3; j++) {
        auto it = cs.rels.find(rel_ids[j]);
        if (it == cs.rels.end()) return false;
        R[j] = it->second.get();
        if (R[j]->nk != 2 || R[j]->attr[0] == R[j]->attr[1]) return false;
    }
    // the attribute relations x and y share, if exactly one
    auto shared = [&](int x, int y, int32_t &a) {
        int n = 0;
        for (int32_t v : R[x]->attr)
            if (std::find(R[y]->attr.begin(), R[y]->attr.end(), v) != R[y]->attr.end()) { a = v; n++; }
        return n == 1;
    };
    int32_t ab = 0, bc = 0, ca = 0;
    if (!shared(0, 1, ab) || !shared(1, 2, bc) || !shared(2, 0, ca)) return false;
    if (ab == bc || bc == ca || ca == ab) return false;
    auto col = [&](int j, int32_t a) {
        return (int)(std::find(R[j]->attr.begin(), R[j]->attr.end(), a) - R[j]->attr.begin());
    };
    q.tri = true;
    // per relation: {shared with the previous one, shared with the next one}
    q.tri_col[0][0] = col(0, ca); q.tri_col[0][1] = col(0, ab);
    q.tri_col[1][0] = col(1, ab); q.tri_col[1][1] = col(1, bc);
    q.tri_col[2][0] = col(2, bc); q.tri_col[2][1] = col(2, ca);
    for (int j = 0; j < 3; j++) {
        q.r[j].rel_id = rel_ids[j];
        q.r[j].R = R[j];
    }
    q.r[0].new_cols = {0, 1};
    q.r[1].parent = 0;
    q.r[1].sep_cols = {col(1, ab)};
    q.r[1].sep_cols_parent = {col(0, ab)};
    q.r[1].new_cols = {col(1, bc)};
    q.r[2].parent = 1;
    q.r[2].sep_cols = {col(2, ca), col(2, bc)};   // factor ordered by (A, C)
    q.r[2].sep_cols_parent = {col(1, bc)};
    q.pre = {0, 1, 2};
    q.pos = {0, 1, 2};
    for (int t = 0; t < 3; t++)
        for (int c : q.r[t].new_cols) { q.var_rel.push_back(t); q.var_col.push_back(c); }
    for (int j = 0; j < 3; j++)
        for (int p = 0; p < R[j]->np; p++) { q.col_rel.push_back(j); q.col_pay.push_back(p); }
    return true;
}

// Plans a query over the relations rel_ids (the first is the root) and gets
// every relation's factor.  Attributes in `drop` are left out of the result
// (early projection, Section 3.7): each must occur in exactly one relation,
// which then groups its rows by its remaining key columns.
gj_status query_create(gj_ctx *ctx, const int32_t *rel_ids, int32_t n_rel,
                       const std::set<int32_t> &drop, gj_query **out) {
    if (!ctx) return GJ_ERR_INVALID;
    std::lock_guard<std::recursive_mutex> lock(ctx->s.mu);
    if (!ctx || !rel_ids || !out || n_rel < 1 || n_rel > MAX_REL) return GJ_ERR_INVALID;
    *out = nullptr;
    for (int32_t a : drop) {
        int holders = 0;
        for (int j = 0; j < n_rel; j++) {
            auto it = ctx->s.rels.find(rel_ids[j]);
            if (it == ctx->s.rels.end()) return GJ_ERR_INVALID;
            const std::vector<int32_t> &attr = it->second->attr;
            holders += (int)std::count(attr.begin(), attr.end(), a);
        }
        // a join attribute would need the potential join of the relations
        // sharing it; an attribute nobody holds is a caller error
        if (holders != 1) return GJ_ERR_INVALID;
    }
    std::unique_ptr<gj_query> qq(new gj_query());
    QueryState &q = qq->s;
    q.cs = &ctx->s;
    q.k = n_rel;
    q.r.resize(n_rel);
    if (n_rel == 3 && drop.empty() && plan_triangle(ctx->s, rel_ids, q)) {
        DeviceGuard g(ctx->s.c.device);
        gj_status st = get_factors(ctx->s, q.r);
        if (st != GJ_OK) return st;
        *out = qq.release();
        return GJ_OK;
    }
    std::set<int32_t> seen;
    for (int j = 0; j < n_rel; j++) {
        auto it = ctx->s.rels.find(rel_ids[j]);
        if (it == ctx->s.rels.end()) return GJ_ERR_INVALID;
        QRel &t = q.r[j];
        t.rel_id = rel_ids[j];
        t.R = it->second.get();
        const std::vector<int32_t> &attr = t.R->attr;
        if (j == 0) {
            for (int c = 0; c < t.R->nk; c++)
                if (!drop.count(attr[c])) t.new_cols.push_back(c);
            if (t.new_cols.empty()) return GJ_ERR_INVALID;   // nothing left to group by
        } else {
            std::vector<int32_t> shared;
            for (int c = 0; c < t.R->nk; c++) {
                if (seen.count(attr[c])) { shared.push_back(attr[c]); t.sep_cols.push_back(c); }
                else if (!drop.count(attr[c])) t.new_cols.push_back(c);
            }
            if (shared.empty()) return GJ_ERR_INVALID;   // a cross product, not an equi-join
            int parent = -1;
            for (int i = 0; i < j && parent < 0; i++) {
                const std::vector<int32_t> &pa = q.r[i].R->attr;
                bool all = true;
                for (int32_t a : shared) all &= std::find(pa.begin(), pa.end(), a) != pa.end();
                if (all) parent = i;
            }
            if (parent < 0) {
                // no join tree in this order: a cyclic query, answered over
                // one maxclique (gj_cyclic.cu), when every relation after the
                // first shares an attribute with those before it
                if (!drop.empty()) return GJ_ERR_NOT_ACYCLIC;
                for (int i = 0; i < n_rel; i++) {
                    auto ri = ctx->s.rels.find(rel_ids[i]);
                    if (ri == ctx->s.rels.end()) return GJ_ERR_INVALID;
                    q.r[i].rel_id = rel_ids[i];
                    q.r[i].R = ri->second.get();
                }
                if (!plan_cyclic(q)) return GJ_ERR_NOT_ACYCLIC;
                DeviceGuard g(ctx->s.c.device);
                gj_status st = get_factors(ctx->s, q.r);
                if (st != GJ_OK) return st;
                *out = qq.release();
                return GJ_OK;
            }
            t.parent = parent;
            const std::vector<int32_t> &pa = q.r[parent].R->attr;
            for (int32_t a : shared)
                t.sep_cols_parent.push_back((int)(std::find(pa.begin(), pa.end(), a) - pa.begin()));
            q.r[parent].children.push_back(j);
        }
        for (int32_t a : attr) seen.insert(a);
    }
    // preorder walk, children in position order
    q.pos.assign(n_rel, -1);
    std::vector<int> stack{0};
    while (!stack.empty()) {
        int t = stack.back();
        stack.pop_back();
        q.pos[t] = (int)q.pre.size();
        q.pre.push_back(t);
        const std::vector<int> &ch = q.r[t].children;
        for (auto it = ch.rbegin(); it != ch.rend(); ++it) stack.push_back(*it);
    }
    for (int t : q.pre)
        for (int c : q.r[t].new_cols) { q.var_rel.push_back(t); q.var_col.push_back(c); }
    for (int j = 0; j < n_rel; j++)
        for (int p = 0; p < q.r[j].R->np; p++) { q.col_rel.push_back(j); q.col_pay.push_back(p); }
    if (q.var_rel.size() > 32 || q.col_rel.size() > 32) return GJ_ERR_INVALID;
    // factors: separator columns lead, then the relation's own columns
    DeviceGuard g(ctx->s.c.device);
    gj_status st = get_factors(ctx->s, q.r);
    if (st != GJ_OK) return st;
    *out = qq.release();
    return GJ_OK;
}

}  // namespace

extern "C" {

gj_status gj_query_create(gj_ctx *ctx, const int32_t *rel_ids, int32_t n_rel, gj_query **out) {
    return query_create(ctx, rel_ids, n_rel, std::set<int32_t>(), out);
}

gj_status gj_query_create_projected(gj_ctx *ctx, const int32_t *rel_ids, int32_t n_rel,
                                    const int32_t *drop_attrs, int32_t n_drop, gj_query **out) {
    if (n_drop < 0 || (n_drop > 0 && !drop_attrs)) return GJ_ERR_INVALID;
    std::set<int32_t> drop(drop_attrs, drop_attrs + n_drop);
    return query_create(ctx, rel_ids, n_rel, drop, out);
}

void gj_query_destroy(gj_query *q) {
    if (!q) return;
    DeviceGuard g(q->s.cs->c.device);
    query_free_summary(q->s.ctx(), q->s);
    for (auto &R : q->s.loaded)
        for (auto &kv : R->factors) factor_free(q->s.ctx(), *kv.second);
    q->s.loaded.clear();
    if (q->s.own) {
        Ctx &o = *q->s.own;
        cudaStreamSynchronize(o.stream);
        cudaFree(o.err);
        cudaFreeHost(o.pinned);
    }
    delete q;
}

gj_status gj_query_set_stream(gj_query *q, void *cuda_stream) {
    if (!q) return GJ_ERR_INVALID;
    QueryState &s = q->s;
    DeviceGuard g(s.cs->c.device);
    if (s.exec && !s.own) return GJ_ERR_STATE;   // runs on a context lent by a server
    if (!s.own) {
        std::unique_ptr<Ctx> o(new Ctx());
        const Ctx &base = s.cs->c;
        o->device = base.device;
        o->pool = base.pool;
        o->num_sms = base.num_sms;
        o->emit_rpt = base.emit_rpt;
        o->tri_mode = base.tri_mode;
        o->down_combine = base.down_combine;
        if (cudaMalloc((void **)&o->err, 16) != cudaSuccess ||
            cudaMallocHost((void **)&o->pinned, 1 << 16) != cudaSuccess) {
            cudaGetLastError();
            if (o->err) cudaFree(o->err);
            return GJ_ERR_OOM;
        }
        cudaMemset(o->err, 0, 16);
        // the query's earlier work (if any) ran on the context's stream
        cudaStreamSynchronize(base.stream);
        s.own = std::move(o);
        s.exec = s.own.get();
    } else {
        cudaStreamSynchronize(s.own->stream);
    }
    s.own->stream = (cudaStream_t)cuda_stream;
    return GJ_OK;
}

gj_status gj_query_sizes(gj_query *q, gj_query_sizes_t *out) {
    if (!q || !out) return GJ_ERR_INVALID;
    memset(out, 0, sizeof(*out));
    QueryState &s = q->s;
    out->n_rel = s.k;
    out->n_vars = (int32_t)s.var_rel.size();
    for (int v = 0; v < out->n_vars; v++) {
        out->var_attr[v] = s.r[s.var_rel[v]].R->attr[s.var_col[v]];
        out->col_width[v] = 4;
    }
    out->n_cols = out->n_vars + (int32_t)s.col_rel.size();
    for (size_t p = 0; p < s.col_rel.size(); p++)
        out->col_width[out->n_vars + p] = s.r[s.col_rel[p]].R->pw[s.col_pay[p]];
    for (int j = 0; j < s.k; j++) {
        out->parent[j] = s.r[j].parent;
        out->n_groups[j] = s.r[j].F->G;
    }
    return GJ_OK;
}

gj_status gj_summarize(gj_query *q, uint64_t *total) {
    if (!q || !total) return GJ_ERR_INVALID;
    if (!q->s.loaded.empty()) {   // a loaded summary is already complete
        *total = q->s.total;
        return q->s.overflow ? GJ_ERR_OVERFLOW : GJ_OK;
    }
    DeviceGuard g(q->s.cs->c.device);
    cudaMemsetAsync(q->s.ctx().err, 0, 4, q->s.ctx().stream);
    return summarize(q->s, total);
}

gj_status gj_summary_groups(gj_query *q, int32_t rel, uint64_t *w_dev, uint64_t *mult_dev,
                            uint64_t *off_dev) {
    if (!q || rel < 0 || rel >= q->s.k || q->s.tri || q->s.cyc) return GJ_ERR_INVALID;
    if (!q->s.summarized && !q->s.overflow) return GJ_ERR_STATE;
    DeviceGuard g(q->s.cs->c.device);
    QRel &t = q->s.r[rel];
    Ctx &c = q->s.ctx();
    size_t bytes = 8 * (size_t)t.F->G;
    if (bytes) {
        if (w_dev && cudaMemcpyAsync(w_dev, t.w, bytes, cudaMemcpyDeviceToDevice, c.stream)) return GJ_ERR_CUDA;
        if (mult_dev && cudaMemcpyAsync(mult_dev, t.mult, bytes, cudaMemcpyDeviceToDevice, c.stream)) return GJ_ERR_CUDA;
        if (off_dev && cudaMemcpyAsync(off_dev, t.off, bytes, cudaMemcpyDeviceToDevice, c.stream)) return GJ_ERR_CUDA;
    }
    return GJ_OK;
}

gj_status gj_level(gj_query *q, int32_t level, uint64_t row0, uint64_t n_rows, int32_t *value_dev,
                   uint64_t *freq_dev, uint64_t *offset_dev, uint64_t cap, uint64_t *n_out) {
    if (!q || !n_out) return GJ_ERR_INVALID;
    DeviceGuard g(q->s.cs->c.device);
    return level_runs(q->s, level, row0, n_rows, value_dev, freq_dev, offset_dev, cap, n_out);
}

gj_status gj_desummarize(gj_query *q, uint64_t row0, uint64_t n_rows, void *const *out_cols,
                         uint32_t *const *rowid_cols, uint64_t *n_out) {
    if (!q || !n_out) return GJ_ERR_INVALID;
    *n_out = 0;
    if (!out_cols) return GJ_ERR_INVALID;
    const int device = q->s.cs->c.device;
    DeviceGuard g(device);
    // every column must be addressable by the device: its own memory,
    // managed memory, or pinned host memory (translated to the device's
    // address for it)
    // (a rejected column is described in gj_last_error)
    auto device_view = [&](void *p, void **dv, const char *what, size_t idx) -> bool {
        cudaPointerAttributes at{};
        cudaError_t e = cudaPointerGetAttributes(&at, p);
        if (e != cudaSuccess) {
            cudaGetLastError();
            snprintf(g_last_error, sizeof(g_last_error), "%s %zu: cudaPointerGetAttributes: %s", what,
                     idx, cudaGetErrorName(e));
            return false;
        }
        if (at.type == cudaMemoryTypeDevice && at.device == device) { *dv = p; return true; }
        if (at.type == cudaMemoryTypeManaged) { *dv = p; return true; }
        if (at.type == cudaMemoryTypeHost && at.devicePointer) { *dv = at.devicePointer; return true; }
        snprintf(g_last_error, sizeof(g_last_error),
                 "%s %zu: memory type %d (device %d, device address %p) is not addressable by device %d",
                 what, idx, (int)at.type, at.device, at.devicePointer, device);
        return false;
    };
    const size_t ncols = q->s.var_rel.size() + q->s.col_rel.size();
    std::vector<void *> cols(ncols);
    for (size_t i = 0; i < ncols; i++) {
        if (!out_cols[i]) {
            snprintf(g_last_error, sizeof(g_last_error), "output column %zu is NULL", i);
            return GJ_ERR_INVALID;
        }
        if (!device_view(out_cols[i], &cols[i], "output column", i)) return GJ_ERR_INVALID;
    }
    std::vector<uint32_t *> rids;
    if (rowid_cols) {
        rids.assign(q->s.k, nullptr);
        for (int j = 0; j < q->s.k; j++) {
            if (!rowid_cols[j]) continue;
            void *dv = nullptr;
            if (!device_view(rowid_cols[j], &dv, "row-id column", (size_t)j)) return GJ_ERR_INVALID;
            rids[j] = (uint32_t *)dv;
        }
    }
    return desummarize(q->s, row0, n_rows, cols.data(), rowid_cols ? rids.data() : nullptr, n_out);
}

}  // extern "C"
