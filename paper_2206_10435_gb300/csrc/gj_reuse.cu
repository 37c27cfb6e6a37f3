// gj_reuse.cu -- compute-and-reuse (Sections 3.6 and 4): store a summary,
// load it later, desummarise from it.
//
// The paper stores the GFJS (one file per column) and later loads and
// desummarises it instead of storing the flat join result.  Here the stored
// object is everything the desummariser reads: per relation the factor
// (row order, group starts, group key values, payloads in group order) and
// the summary arrays (segments, links, w, offsets, messages, multiplicities,
// live groups), plus the join tree and output layout.  Its size is
// O(input + groups); the result it reproduces is O(|Q|).  A loaded summary
// is a query of its own: it owns its device copies and needs none of the
// original relations.
//
// File layout: a fixed header (magic, version, sizes) followed by records
// (tag, byte count, bytes) in a fixed order; all integers little-endian as
// in memory.
#include <stdio.h>
#include <string.h>

#include <memory>

#include "gj_state.cuh"

namespace gj {

void query_free_summary(Ctx &c, QueryState &q);
void factor_free(Ctx &c, Factor &F);

namespace {

constexpr char MAGIC[8] = {'G', 'J', 'S', 'U', 'M', 'M', '0', '1'};

struct Writer {
    FILE *f;
    Ctx &c;
    uint64_t bytes = 0;
    bool ok = true;
    std::vector<char> host;
    void raw(const void *p, size_t n) {
        if (ok && n && fwrite(p, 1, n, f) != n) ok = false;
        bytes += n;
    }
    template <class T>
    void val(T v) { raw(&v, sizeof(T)); }
    template <class T>
    void vec(const std::vector<T> &v) {
        val<uint64_t>(v.size());
        raw(v.data(), v.size() * sizeof(T));
    }
    // device array of n elements
    template <class T>
    void dev(const T *p, uint64_t n) {
        val<uint64_t>(n);
        if (!n) return;
        host.resize(n * sizeof(T));
        if (cudaMemcpyAsync(host.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
            cudaStreamSynchronize(c.stream) != cudaSuccess) {
            ok = false;
            return;
        }
        raw(host.data(), n * sizeof(T));
    }
};

struct Reader {
    FILE *f;
    Ctx &c;
    bool ok = true;
    std::vector<char> host;
    void raw(void *p, size_t n) {
        if (ok && n && fread(p, 1, n, f) != n) ok = false;
    }
    template <class T>
    T val() {
        T v{};
        raw(&v, sizeof(T));
        return v;
    }
    template <class T>
    std::vector<T> vec() {
        uint64_t n = val<uint64_t>();
        std::vector<T> v;
        if (!ok || n > (1ull << 40)) { ok = false; return v; }
        v.resize(n);
        raw(v.data(), n * sizeof(T));
        return v;
    }
    // allocates a device array and fills it; returns the element count
    template <class T>
    uint64_t dev(T **p) {
        uint64_t n = val<uint64_t>();
        *p = nullptr;
        if (!ok || n > (1ull << 40)) { ok = false; return 0; }
        if (dalloc(c, p, n) != cudaSuccess) { ok = false; return 0; }
        if (!n) return 0;
        host.resize(n * sizeof(T));
        raw(host.data(), n * sizeof(T));
        if (ok && (cudaMemcpyAsync(*p, host.data(), n * sizeof(T), cudaMemcpyHostToDevice, c.stream) != cudaSuccess ||
                   cudaStreamSynchronize(c.stream) != cudaSuccess))
            ok = false;
        return n;
    }
};

uint32_t read_u32(Ctx &c, const uint32_t *p) {
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, p, 4, cudaMemcpyDeviceToHost, c.stream) == cudaSuccess)
        cudaStreamSynchronize(c.stream);
    return v;
}

}  // namespace
}  // namespace gj

using namespace gj;

extern "C" {

gj_status gj_summary_save(gj_query *qq, const char *path, uint64_t *bytes) {
    if (!qq || !path || qq->s.tri || qq->s.cyc) return GJ_ERR_INVALID;
    QueryState &q = qq->s;
    if (!q.summarized) return GJ_ERR_STATE;
    Ctx &c = q.ctx();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c.device);
    FILE *f = fopen(path, "wb");
    if (!f) { if (prev >= 0) cudaSetDevice(prev); return GJ_ERR_INVALID; }
    Writer w{f, c};
    w.raw(MAGIC, 8);
    w.val<int32_t>(q.k);
    w.val<uint64_t>(q.total);
    w.val<int32_t>(q.overflow ? 1 : 0);
    w.vec(q.pre);
    w.vec(q.pos);
    w.vec(q.var_rel);
    w.vec(q.var_col);
    w.vec(q.col_rel);
    w.vec(q.col_pay);
    for (int j = 0; j < q.k && w.ok; j++) {
        const QRel &t = q.r[j];
        const Relation &R = *t.R;
        const Factor &F = *t.F;
        w.val<int64_t>(R.n);
        w.val<int32_t>(R.nk);
        w.val<int32_t>(R.np);
        w.vec(R.attr);
        w.vec(R.pw);
        w.val<int32_t>(t.parent);
        w.vec(t.children);
        w.vec(t.sep_cols);
        w.vec(t.sep_cols_parent);
        w.vec(t.new_cols);
        w.vec(F.order);
        w.val<int64_t>(F.G);
        w.dev(F.perm, (uint64_t)R.n);
        w.dev(F.gstart, (uint64_t)F.G + 1);
        w.dev(F.gkey, (uint64_t)R.nk * F.G);
        for (int p = 0; p < R.np; p++) {
            if (R.pw[p] == 8) w.dev((const uint64_t *)F.pay[p], (uint64_t)R.n);
            else w.dev((const uint32_t *)F.pay[p], (uint64_t)R.n);
        }
        const uint64_t G = (uint64_t)F.G;
        const uint64_t S = t.parent >= 0 ? read_u32(c, t.S_dev) : 0;
        const uint64_t L = read_u32(c, t.L_dev);
        w.val<uint64_t>(S);
        w.val<uint64_t>(L);
        if (t.parent >= 0) {
            w.dev(t.seg_id, G);
            w.dev(t.seg_first, S + 1);
            w.dev(t.msg, S);
            w.dev(t.down, S);
            w.dev(t.lseg_first, S + 1);
        }
        for (size_t ci = 0; ci < t.children.size(); ci++) w.dev(t.link[ci], G);
        w.dev(t.w, G);
        w.dev(t.off, G);
        w.dev(t.mult, G);
        w.dev(t.lgid, L);
        w.dev(t.loff, L);
        w.dev(t.lw, L);
    }
    w.raw(MAGIC, 8);
    bool ok = w.ok;
    if (fclose(f) != 0) ok = false;
    if (prev >= 0) cudaSetDevice(prev);
    if (bytes) *bytes = w.bytes;
    return ok ? GJ_OK : GJ_ERR_CUDA;
}

gj_status gj_summary_load(gj_ctx *ctx, const char *path, gj_query **out) {
    if (!ctx || !path || !out) return GJ_ERR_INVALID;
    *out = nullptr;
    Ctx &c = ctx->s.c;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c.device);
    FILE *f = fopen(path, "rb");
    if (!f) { if (prev >= 0) cudaSetDevice(prev); return GJ_ERR_INVALID; }
    std::unique_ptr<gj_query> qq(new gj_query());
    QueryState &q = qq->s;
    q.cs = &ctx->s;
    Reader r{f, c};
    char magic[8];
    r.raw(magic, 8);
    bool ok = r.ok && memcmp(magic, MAGIC, 8) == 0;
    if (ok) {
        q.k = r.val<int32_t>();
        q.total = r.val<uint64_t>();
        q.overflow = r.val<int32_t>() != 0;
        ok = r.ok && q.k >= 1 && q.k <= MAX_REL;
    }
    if (ok) {
        q.pre = r.vec<int>();
        q.pos = r.vec<int>();
        q.var_rel = r.vec<int>();
        q.var_col = r.vec<int>();
        q.col_rel = r.vec<int>();
        q.col_pay = r.vec<int>();
        q.r.resize(q.k);
        ok = r.ok && (int)q.pre.size() == q.k && (int)q.pos.size() == q.k;
    }
    for (int j = 0; j < q.k && ok; j++) {
        QRel &t = q.r[j];
        std::unique_ptr<Relation> R(new Relation());
        std::unique_ptr<Factor> F(new Factor());
        R->n = r.val<int64_t>();
        R->nk = r.val<int32_t>();
        R->np = r.val<int32_t>();
        R->attr = r.vec<int32_t>();
        R->pw = r.vec<int32_t>();
        t.parent = r.val<int32_t>();
        t.children = r.vec<int>();
        t.sep_cols = r.vec<int>();
        t.sep_cols_parent = r.vec<int>();
        t.new_cols = r.vec<int>();
        F->order = r.vec<int>();
        F->G = r.val<int64_t>();
        F->n = R->n;
        if (!r.ok || R->nk < 1 || R->nk > MAX_KEYS || R->np < 0 || R->np > MAX_PAYLOADS ||
            (int)R->attr.size() != R->nk || (int)R->pw.size() != R->np) { ok = false; break; }
        r.dev(&F->perm);
        r.dev(&F->gstart);
        r.dev(&F->gkey);
        for (int p = 0; p < R->np; p++) {
            void *d = nullptr;
            if (R->pw[p] == 8) { uint64_t *x; r.dev(&x); d = x; }
            else { uint32_t *x; r.dev(&x); d = x; }
            F->pay.push_back(d);
        }
        const uint64_t S = r.val<uint64_t>();
        const uint64_t L = r.val<uint64_t>();
        if (t.parent >= 0) {
            r.dev(&t.seg_id);
            r.dev(&t.seg_first);
            r.dev(&t.msg);
            r.dev(&t.down);
            r.dev(&t.lseg_first);
        }
        t.link.assign(t.children.size(), nullptr);
        for (size_t ci = 0; ci < t.children.size(); ci++) r.dev(&t.link[ci]);
        r.dev(&t.w);
        r.dev(&t.off);
        r.dev(&t.mult);
        r.dev(&t.lgid);
        r.dev(&t.loff);
        r.dev(&t.lw);
        // counts back into device memory
        if (dalloc(c, &t.S_dev, 1) != cudaSuccess || dalloc(c, &t.L_dev, 1) != cudaSuccess) { ok = false; break; }
        uint32_t sl[2] = {(uint32_t)S, (uint32_t)L};
        if (cudaMemcpyAsync(t.S_dev, &sl[0], 4, cudaMemcpyHostToDevice, c.stream) != cudaSuccess ||
            cudaMemcpyAsync(t.L_dev, &sl[1], 4, cudaMemcpyHostToDevice, c.stream) != cudaSuccess ||
            cudaStreamSynchronize(c.stream) != cudaSuccess) { ok = false; break; }
        R->have_minmax = true;
        R->kmin.assign(R->nk, 0);
        R->kmax.assign(R->nk, 0);
        t.F = F.get();
        t.R = R.get();
        t.rel_id = -1;
        R->factors[F->order] = std::move(F);
        q.loaded.push_back(std::move(R));
        ok = r.ok;
    }
    if (ok) {
        r.raw(magic, 8);
        ok = r.ok && memcmp(magic, MAGIC, 8) == 0;
    }
    fclose(f);
    if (!ok) {
        query_free_summary(c, q);
        for (auto &R : q.loaded)
            for (auto &kv : R->factors) factor_free(c, *kv.second);
        if (prev >= 0) cudaSetDevice(prev);
        return r.ok ? GJ_ERR_INVALID : GJ_ERR_INVALID;
    }
    q.summarized = true;
    if (prev >= 0) cudaSetDevice(prev);
    *out = qq.release();
    return GJ_OK;
}

}  // extern "C"
