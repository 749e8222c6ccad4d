// C ABI of libgofmm (include/gofmm.h): argument checks, error codes, handle
// ownership, checkpoint files and structure views.  All work is delegated to
// compress.cpp (host) and eval.cu (device).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <memory>
#include <new>

#include "gofmm_internal.hpp"

struct gofmm_handle {
    gofmm::Handle h;
};

struct gofmm_engine {
    gofmm::Engine* e = nullptr;
};

struct gofmm_batch {
    gofmm::Batch* b = nullptr;
    int last_launches = 0;
};

namespace {
thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

template <class F>
int guarded(F&& f) {
    try {
        g_last_error.clear();
        f();
        return GOFMM_OK;
    } catch (const gofmm::Error& e) {
        return set_error(e.code, e.msg);
    } catch (const std::bad_alloc&) {
        return set_error(GOFMM_ERR_NOMEM, "host allocation failed");
    } catch (const std::exception& e) {
        return set_error(GOFMM_ERR_ARG, e.what());
    }
}

void check_entries(const gofmm_entries* K) {
    using gofmm::fail;
    if (!K) fail(GOFMM_ERR_ARG, "entries is NULL");
    if (K->n < 1) fail(GOFMM_ERR_ARG, "n must be >= 1");
    if (K->kind == GOFMM_GEN_CALLBACK) {
        if (!K->fn) fail(GOFMM_ERR_ARG, "callback kind needs fn");
    } else if (K->kind == GOFMM_GEN_GAUSSIAN || K->kind == GOFMM_GEN_IMQ) {
        if (!K->points || K->dim < 1) fail(GOFMM_ERR_ARG, "generator kind needs points and dim >= 1");
        if (!(K->bandwidth > 0) || !std::isfinite(K->diag_shift)) fail(GOFMM_ERR_ARG, "bandwidth must be > 0");
    } else {
        fail(GOFMM_ERR_ARG, "unknown entries kind");
    }
}

gofmm::Entries make_entries(const gofmm_entries* K) {
    gofmm::Entries E;
    E.kind = K->kind;
    E.n = K->n;
    E.dim = K->dim;
    E.h = K->bandwidth;
    E.shift = K->diag_shift;
    E.fn = K->fn;
    E.ctx = K->ctx;
    if (E.is_generator()) {
        E.pts.assign(K->points, K->points + size_t(K->n) * size_t(K->dim));
        for (double v : E.pts)
            if (!std::isfinite(v)) gofmm::fail(GOFMM_ERR_NONFINITE, "non-finite point coordinate");
    }
    return E;
}

gofmm::Params make_params(const gofmm_params* p) {
    using gofmm::fail;
    gofmm::Params q;
    q.m = p->leaf_size;
    q.s = p->max_rank;
    q.tau = p->tau;
    q.budget = p->budget;
    q.kappa = p->kappa;
    q.distance = p->distance;
    q.far_mode = p->far_mode;
    q.cache_mode = p->cache_mode;
    q.n_centroid = p->n_centroid;
    q.n_sample = p->n_sample;
    q.ann_max_iter = p->ann_max_iter;
    q.num_threads = p->num_threads;
    q.ann_target_recall = p->ann_target_recall;
    q.knn_exact_max = p->knn_exact_max;
    q.seed = p->seed;
    q.device = p->device;
    q.sample_device = p->sample_device;
    if (q.sample_device != 0 && q.sample_device != 1) fail(GOFMM_ERR_ARG, "sample_device must be 0 or 1");
    if (q.m < 1) fail(GOFMM_ERR_ARG, "leaf_size must be >= 1");
    if (q.s < 1) fail(GOFMM_ERR_ARG, "max_rank must be >= 1");
    if (!(q.tau >= 0)) fail(GOFMM_ERR_ARG, "tau must be >= 0");
    if (!(q.budget >= 0)) fail(GOFMM_ERR_ARG, "budget must be >= 0");
    if (q.kappa < 1) fail(GOFMM_ERR_ARG, "kappa must be >= 1");
    if (q.n_centroid < 1) fail(GOFMM_ERR_ARG, "n_centroid must be >= 1");
    if (q.n_sample < 0 || q.ann_max_iter < 1) fail(GOFMM_ERR_ARG, "n_sample >= 0 and ann_max_iter >= 1");
    if (q.distance < GOFMM_DIST_GRAM_L2 || q.distance > GOFMM_DIST_RANDOM) fail(GOFMM_ERR_ARG, "unknown distance");
    if (q.far_mode != GOFMM_FAR_SYMMETRIC && q.far_mode != GOFMM_FAR_PAPER) fail(GOFMM_ERR_ARG, "unknown far_mode");
    if (q.cache_mode != GOFMM_CACHE_BLOCKS && q.cache_mode != GOFMM_CACHE_NONE) fail(GOFMM_ERR_ARG, "unknown cache_mode");
    return q;
}

// ---- checkpoint file ------------------------------------------------------
const char kMagic[8] = {'G', 'O', 'F', 'M', 'M', 'S', 'T', '1'};

struct Writer {
    std::ofstream f;
    template <class T>
    void put(const T& v) { f.write(reinterpret_cast<const char*>(&v), sizeof(T)); }
    template <class T>
    void vec(const std::vector<T>& v) {
        put<int64_t>(int64_t(v.size()));
        if (!v.empty()) f.write(reinterpret_cast<const char*>(v.data()), std::streamsize(v.size() * sizeof(T)));
    }
};
struct Reader {
    std::ifstream f;
    template <class T>
    T get() {
        T v;
        f.read(reinterpret_cast<char*>(&v), sizeof(T));
        if (!f) gofmm::fail(GOFMM_ERR_IO, "truncated structure file");
        return v;
    }
    template <class T>
    std::vector<T> vec(int64_t limit) {
        const int64_t n = get<int64_t>();
        if (n < 0 || n > limit) gofmm::fail(GOFMM_ERR_IO, "corrupt structure file");
        std::vector<T> v(static_cast<size_t>(n));
        if (n) f.read(reinterpret_cast<char*>(v.data()), std::streamsize(n * sizeof(T)));
        if (!f) gofmm::fail(GOFMM_ERR_IO, "truncated structure file");
        return v;
    }
};
}  // namespace

namespace gofmm {
void export_structure(const Structure& st, const Entries*, const std::string& path) {
    Writer w;
    w.f.open(path, std::ios::binary);
    if (!w.f) fail(GOFMM_ERR_IO, "cannot open " + path + " for writing");
    w.f.write(kMagic, 8);
    const Params& p = st.prm;
    w.put<int64_t>(st.n);
    w.put<int64_t>(st.depth);
    w.put(p.m); w.put(p.s); w.put(p.tau); w.put(p.budget);
    w.put<int64_t>(p.kappa); w.put<int64_t>(p.distance); w.put<int64_t>(p.far_mode);
    w.put<uint64_t>(p.seed);
    w.put<int64_t>(st.ann_iters); w.put(st.ann_recall);
    w.vec(st.perm);
    w.vec(st.node_size);
    for (const auto& v : st.near) w.vec(v);
    for (const auto& v : st.far) w.vec(v);
    for (const auto& v : st.skel) w.vec(v);
    for (const auto& v : st.P) w.vec(v);
    if (!w.f) fail(GOFMM_ERR_IO, "write failed: " + path);
}

void import_structure(const std::string& path, Structure& st) {
    Reader r;
    r.f.open(path, std::ios::binary);
    if (!r.f) fail(GOFMM_ERR_IO, "cannot open " + path);
    char mg[8];
    r.f.read(mg, 8);
    if (!r.f || std::memcmp(mg, kMagic, 8) != 0) fail(GOFMM_ERR_IO, "not a GOFMM structure file");
    st.n = r.get<int64_t>();
    st.depth = int(r.get<int64_t>());
    if (st.n < 1 || st.depth < 0 || st.depth > 40 || (int64_t(1) << st.depth) > st.n)
        fail(GOFMM_ERR_IO, "corrupt structure header");
    Params& p = st.prm;
    p.m = r.get<int64_t>(); p.s = r.get<int64_t>(); p.tau = r.get<double>(); p.budget = r.get<double>();
    p.kappa = int(r.get<int64_t>()); p.distance = int(r.get<int64_t>()); p.far_mode = int(r.get<int64_t>());
    p.seed = r.get<uint64_t>();
    st.ann_iters = int(r.get<int64_t>()); st.ann_recall = r.get<double>();
    const int64_t nn = st.n_nodes(), nl = st.n_leaves();
    st.perm = r.vec<int64_t>(st.n);
    st.node_size = r.vec<int64_t>(nn);
    if (int64_t(st.perm.size()) != st.n || int64_t(st.node_size.size()) != nn) fail(GOFMM_ERR_IO, "corrupt structure");
    std::vector<char> seen(st.n, 0);
    for (int64_t i : st.perm) {
        if (i < 0 || i >= st.n || seen[i]) fail(GOFMM_ERR_IO, "perm is not a permutation");
        seen[i] = 1;
    }
    int64_t total = 0;
    for (int64_t b = 0; b < nl; ++b) total += st.node_size[st.leaf_node(b)];
    if (total != st.n) fail(GOFMM_ERR_IO, "leaf sizes do not add up to n");
    fill_node_extents(st);
    st.near.resize(nl);
    for (auto& v : st.near) {
        v = r.vec<int64_t>(nl);
        for (int64_t a : v) if (a < 0 || a >= nl) fail(GOFMM_ERR_IO, "bad near list");
    }
    st.far.resize(nn);
    for (auto& v : st.far) {
        v = r.vec<int64_t>(nn);
        for (int64_t a : v) if (a < 1 || a >= nn) fail(GOFMM_ERR_IO, "bad far list");
    }
    st.skel.resize(nn);
    for (int64_t h = 0; h < nn; ++h) {
        st.skel[h] = r.vec<int64_t>(st.n);
        for (int64_t a : st.skel[h]) if (a < 0 || a >= st.n) fail(GOFMM_ERR_IO, "bad skeleton");
        if ((h == 0) != st.skel[h].empty()) fail(GOFMM_ERR_IO, "skeleton presence mismatch");
    }
    st.P.resize(nn);
    for (int64_t h = 0; h < nn; ++h) {
        st.P[h] = r.vec<double>(int64_t(1) << 40);
        const int64_t want = h == 0 ? 0 : int64_t(st.skel[h].size()) * st.ncols(h);
        if (int64_t(st.P[h].size()) != want) fail(GOFMM_ERR_IO, "interpolation matrix size mismatch");
    }
}
}  // namespace gofmm

extern "C" {

void gofmm_default_params(gofmm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->leaf_size = 64;
    p->max_rank = 64;
    p->tau = 1e-5;
    p->budget = 0.03;
    p->kappa = 32;
    p->distance = GOFMM_DIST_GRAM_L2;
    p->far_mode = GOFMM_FAR_SYMMETRIC;
    p->cache_mode = GOFMM_CACHE_BLOCKS;
    p->n_centroid = 32;
    p->n_sample = 0;
    p->ann_max_iter = 10;
    p->num_threads = 0;
    p->ann_target_recall = 0.8;
    p->knn_exact_max = 16384;
    p->seed = 0;
    p->device = 0;
}

const char* gofmm_last_error(void) { return g_last_error.c_str(); }

int gofmm_compress(const gofmm_entries* K, const gofmm_params* p, gofmm_handle** out) {
    if (out) *out = nullptr;
    return guarded([&] {
        if (!out) gofmm::fail(GOFMM_ERR_ARG, "out is NULL");
        check_entries(K);
        gofmm_params d;
        gofmm_default_params(&d);
        auto h = std::make_unique<gofmm_handle>();
        h->h.st.prm = make_params(p ? p : &d);
        if (h->h.st.prm.cache_mode == GOFMM_CACHE_NONE && K->kind == GOFMM_GEN_CALLBACK)
            gofmm::fail(GOFMM_ERR_ARG, "CACHE_NONE needs a generator kind (entries are made in-kernel)");
        h->h.K = make_entries(K);
        gofmm::compress(h->h.K, h->h.st);
        h->h.K.fn = nullptr;  // the callback is not kept past this call
        h->h.K.ctx = nullptr;
        *out = h.release();
    });
}

int gofmm_prepare(gofmm_handle* h, int64_t r_max, int precision) {
    return guarded([&] {
        if (!h) gofmm::fail(GOFMM_ERR_ARG, "handle is NULL");
        gofmm::device_prepare(h->h, r_max, precision);
    });
}

int gofmm_evaluate(gofmm_handle* h, const void* W, int64_t ldw, void* U, int64_t ldu, int64_t r,
                   int dtype, int precision, void* stream) {
    return guarded([&] {
        if (!h) gofmm::fail(GOFMM_ERR_ARG, "handle is NULL");
        gofmm::device_evaluate(h->h, W, ldw, U, ldu, r, dtype, precision, stream, 0);
    });
}

int gofmm_evaluate_host(gofmm_handle* h, const void* W, int64_t ldw, void* U, int64_t ldu, int64_t r,
                        int dtype, int precision, void* stream) {
    return guarded([&] {
        if (!h) gofmm::fail(GOFMM_ERR_ARG, "handle is NULL");
        gofmm::device_evaluate(h->h, W, ldw, U, ldu, r, dtype, precision, stream, 1);
    });
}

int gofmm_evaluate_host_async(gofmm_handle* h, const void* W, int64_t ldw, void* U, int64_t ldu, int64_t r,
                              int dtype, int precision, void* stream) {
    return guarded([&] {
        if (!h) gofmm::fail(GOFMM_ERR_ARG, "handle is NULL");
        gofmm::device_evaluate(h->h, W, ldw, U, ldu, r, dtype, precision, stream, 2);
    });
}

int gofmm_evaluate_static(gofmm_handle* h, const void* W, int64_t ldw, void* U, int64_t ldu, int64_t r,
                          int dtype, int precision, void* stream) {
    return guarded([&] {
        if (!h) gofmm::fail(GOFMM_ERR_ARG, "handle is NULL");
        gofmm::device_evaluate_static(h->h, W, ldw, U, ldu, r, dtype, precision, stream);
    });
}

int gofmm_debug_stall_next(gofmm_handle* h, int precision) {
    return guarded([&] {
        if (!h) gofmm::fail(GOFMM_ERR_ARG, "handle is NULL");
        gofmm::device_stall_next(h->h, precision);
    });
}

int gofmm_set_tc_config(gofmm_handle* h, int precision, int piece, int schedule, int order) {
    return guarded([&] {
        if (!h) gofmm::fail(GOFMM_ERR_ARG, "handle is NULL");
        gofmm::device_set_tc_config(h->h, precision, piece, schedule, order);
    });
}

int gofmm_get_tc_config(const gofmm_handle* h, int precision, int* piece, int* schedule, int* order) {
    return guarded([&] {
        if (!h) gofmm::fail(GOFMM_ERR_ARG, "handle is NULL");
        if (precision != GOFMM_PREC_TF32 && precision != GOFMM_PREC_BF16 && precision != GOFMM_PREC_BF16X3)
            gofmm::fail(GOFMM_ERR_ARG, "the launch configuration belongs to a tensor-core precision");
        const int mode = precision == GOFMM_PREC_TF32 ? 0 : precision == GOFMM_PREC_BF16 ? 1 : 2;
        if (piece) *piece = h->h.tc_piece[mode];
        if (schedule) *schedule = h->h.tc_schedule[mode];
        if (order) *order = h->h.tc_order[mode];
    });
}

namespace {
void fill_tune(const gofmm::TuneResult& t, gofmm_tune_t* out) {
    if (!out) return;
    std::memset(out, 0, sizeof *out);
    out->piece = t.piece;
    out->schedule = t.schedule;
    out->order = t.order;
    out->from_cache = t.from_cache;
    out->n_candidates = t.n;
    for (int k = 0; k < t.n && k < 16; ++k) {
        out->cand_piece[k] = t.cand_piece[k];
        out->cand_schedule[k] = t.cand_schedule[k];
        out->cand_order[k] = t.cand_order[k];
        out->cand_ms[k] = t.cand_ms[k];
    }
    std::snprintf(out->key, sizeof out->key, "%s", t.key.c_str());
}
}  // namespace

int gofmm_autotune(gofmm_handle* h, int64_t r, int precision, const char* cache_path, void* stream,
                   gofmm_tune_t* out) {
    return guarded([&] {
        if (!h) gofmm::fail(GOFMM_ERR_ARG, "handle is NULL");
        fill_tune(gofmm::autotune(h->h, r, precision, cache_path, stream), out);
    });
}

int gofmm_autotune_batch(gofmm_handle* const* hs, const int64_t* r, int count, int precision,
                         const char* cache_path, void* stream, gofmm_tune_t* out) {
    return guarded([&] {
        if (!hs || !r || count < 1) gofmm::fail(GOFMM_ERR_ARG, "need count >= 1 handles and r values");
        std::vector<gofmm::Handle*> v;
        for (int i = 0; i < count; ++i) {
            if (!hs[i]) gofmm::fail(GOFMM_ERR_ARG, "NULL handle");
            v.push_back(&hs[i]->h);
        }
        fill_tune(gofmm::autotune_batch(v.data(), r, count, precision, cache_path, stream), out);
    });
}

int gofmm_autotune_key(gofmm_handle* const* hs, const int64_t* r, int count, int precision, char* key) {
    return guarded([&] {
        if (!hs || !r || count < 1 || !key) gofmm::fail(GOFMM_ERR_ARG, "need handles, r values and a key buffer");
        std::vector<gofmm::Handle*> v;
        for (int i = 0; i < count; ++i) {
            if (!hs[i]) gofmm::fail(GOFMM_ERR_ARG, "NULL handle");
            v.push_back(&hs[i]->h);
        }
        std::snprintf(key, 32, "%s", gofmm::tune_key_batch(v.data(), r, count, precision).c_str());
    });
}

int gofmm_trim(gofmm_handle* h) {
    return guarded([&] {
        if (!h) gofmm::fail(GOFMM_ERR_ARG, "handle is NULL");
        gofmm::device_trim(h->h);
    });
}

int gofmm_synchronize(gofmm_handle* h, void* stream) {
    return guarded([&] {
        if (!h) gofmm::fail(GOFMM_ERR_ARG, "handle is NULL");
        gofmm::device_synchronize(h->h, stream);
    });
}

int gofmm_engine_create(int device, int precision, int64_t pool_bytes, gofmm_engine** out) {
    if (out) *out = nullptr;
    return guarded([&] {
        if (!out) gofmm::fail(GOFMM_ERR_ARG, "out is NULL");
        auto w = std::make_unique<gofmm_engine>();
        w->e = gofmm::engine_create(device, precision, pool_bytes);
        *out = w.release();
    });
}

int gofmm_engine_submit(gofmm_engine* e, gofmm_handle* h, const void* W, int64_t ldw, void* U, int64_t ldu,
                        int64_t r, int64_t* id) {
    return guarded([&] {
        if (!e || !h || !id) gofmm::fail(GOFMM_ERR_ARG, "engine, handle and id must not be NULL");
        *id = gofmm::engine_submit(*e->e, h->h, static_cast<const float*>(W), ldw, static_cast<float*>(U), ldu, r);
    });
}

int gofmm_engine_step(gofmm_engine* e, void* stream, int64_t* pending) {
    return guarded([&] {
        if (!e) gofmm::fail(GOFMM_ERR_ARG, "engine is NULL");
        const int64_t n = gofmm::engine_step(*e->e, static_cast<cudaStream_t>(stream));
        if (pending) *pending = n;
    });
}

int gofmm_engine_workspace(const gofmm_engine* e, gofmm_handle* h, int64_t r, int64_t* bytes) {
    return guarded([&] {
        if (!e || !h || !bytes) gofmm::fail(GOFMM_ERR_ARG, "engine, handle and bytes must not be NULL");
        *bytes = gofmm::engine_workspace(*e->e, h->h, r);
    });
}

int gofmm_engine_poll(gofmm_engine* e, int64_t id, int* state) {
    return guarded([&] {
        if (!e || !state) gofmm::fail(GOFMM_ERR_ARG, "engine and state must not be NULL");
        *state = gofmm::engine_poll(*e->e, id);
    });
}

int gofmm_engine_drain(gofmm_engine* e, void* stream) {
    return guarded([&] {
        if (!e) gofmm::fail(GOFMM_ERR_ARG, "engine is NULL");
        gofmm::engine_drain(*e->e, static_cast<cudaStream_t>(stream));
    });
}

int gofmm_engine_stats(const gofmm_engine* e, int64_t* out, int n) {
    return guarded([&] {
        if (!e || !out || n < 1) gofmm::fail(GOFMM_ERR_ARG, "bad arguments");
        gofmm::engine_stats(*e->e, out, n);
    });
}

int gofmm_engine_free(gofmm_engine* e) {
    if (!e) return GOFMM_OK;
    int rc = guarded([&] { gofmm::engine_destroy(e->e); });
    delete e;
    return rc;
}

int gofmm_batch_create(gofmm_handle* const* hs, const int64_t* r, int count, int precision, gofmm_batch** out) {
    if (out) *out = nullptr;
    return guarded([&] {
        if (!out || !hs || !r || count < 1) gofmm::fail(GOFMM_ERR_ARG, "bad batch arguments");
        std::vector<gofmm::Handle*> hv;
        for (int i = 0; i < count; ++i) {
            if (!hs[i]) gofmm::fail(GOFMM_ERR_ARG, "NULL handle in batch");
            hv.push_back(&hs[i]->h);
        }
        auto w = std::make_unique<gofmm_batch>();
        w->b = gofmm::batch_create(hv.data(), r, count, precision);
        *out = w.release();
    });
}

int gofmm_batch_evaluate(gofmm_batch* b, const void* const* W, const int64_t* ldw, void* const* U,
                         const int64_t* ldu, void* stream) {
    return guarded([&] {
        if (!b || !W || !ldw || !U || !ldu) gofmm::fail(GOFMM_ERR_ARG, "bad batch arguments");
        b->last_launches = gofmm::batch_evaluate(*b->b, reinterpret_cast<const float* const*>(W), ldw,
                                                 reinterpret_cast<float* const*>(U), ldu,
                                                 static_cast<cudaStream_t>(stream));
    });
}

int gofmm_batch_info(const gofmm_batch* b, int64_t* out, int n) {
    return guarded([&] {
        if (!b || !out || n < 1) gofmm::fail(GOFMM_ERR_ARG, "bad arguments");
        const int64_t v[2] = {int64_t(b->last_launches), int64_t(gofmm::batch_error(*b->b))};
        for (int i = 0; i < n && i < 2; ++i) out[i] = v[i];
    });
}

int gofmm_batch_free(gofmm_batch* b) {
    if (!b) return GOFMM_OK;
    int rc = guarded([&] { gofmm::batch_destroy(b->b); });
    delete b;
    return rc;
}

int gofmm_free(gofmm_handle* h) {
    if (!h) return GOFMM_OK;
    if (h->h.inflight > 0)
        return set_error(GOFMM_ERR_ARG, "a serving engine holds requests of this handle: drain the engine first");
    int rc = guarded([&] { gofmm::device_destroy(h->h); });
    delete h;
    return rc;
}

int gofmm_export(const gofmm_handle* h, const char* path) {
    return guarded([&] {
        if (!h || !path) gofmm::fail(GOFMM_ERR_ARG, "handle or path is NULL");
        gofmm::export_structure(h->h.st, &h->h.K, path);
    });
}

int gofmm_import(const char* path, const gofmm_entries* K, int cache_mode, int device, gofmm_handle** out) {
    if (out) *out = nullptr;
    return guarded([&] {
        if (!out || !path) gofmm::fail(GOFMM_ERR_ARG, "path or out is NULL");
        check_entries(K);
        auto h = std::make_unique<gofmm_handle>();
        gofmm::import_structure(path, h->h.st);
        if (K->n != h->h.st.n) gofmm::fail(GOFMM_ERR_ARG, "entries describe a different N");
        if (cache_mode != GOFMM_CACHE_BLOCKS && cache_mode != GOFMM_CACHE_NONE)
            gofmm::fail(GOFMM_ERR_ARG, "unknown cache_mode");
        if (cache_mode == GOFMM_CACHE_NONE && K->kind == GOFMM_GEN_CALLBACK)
            gofmm::fail(GOFMM_ERR_ARG, "CACHE_NONE needs a generator kind");
        h->h.st.prm.cache_mode = cache_mode;
        h->h.st.prm.device = device;
        h->h.K = make_entries(K);
        if (!h->h.K.is_generator() && cache_mode == GOFMM_CACHE_BLOCKS) gofmm::cache_blocks_host(h->h.K, h->h.st);
        h->h.K.fn = nullptr;
        h->h.K.ctx = nullptr;
        *out = h.release();
    });
}

int gofmm_stats(const gofmm_handle* hd, gofmm_stats_t* s) {
    return guarded([&] {
        if (!hd || !s) gofmm::fail(GOFMM_ERR_ARG, "handle or stats is NULL");
        const gofmm::Structure& st = hd->h.st;
        std::memset(s, 0, sizeof(*s));
        s->n = st.n;
        s->depth = st.depth;
        s->n_leaves = st.n_leaves();
        s->min_rank = INT64_MAX;
        int64_t cnt = 0;
        for (int64_t h = 1; h < st.n_nodes(); ++h) {
            const int64_t r = int64_t(st.skel[h].size());
            s->min_rank = std::min(s->min_rank, r);
            s->max_rank = std::max(s->max_rank, r);
            s->skel_total += r;
            s->interp_entries += int64_t(st.P[h].size());
            // P = [I | T] Pi^T: only the T part (s x (ncols - s)) is
            // arithmetic; the identity part is a copy (Table 2, real shapes)
            const int64_t t_entries = int64_t(st.P[h].size()) - r * r;
            s->interp_t_entries += t_entries;
            ++cnt;
            s->flops_n2s += 2.0 * double(t_entries);
            for (int64_t a : st.far[h]) {
                s->flops_s2s += 2.0 * double(r) * double(st.skel[a].size());
                s->far_entries += r * int64_t(st.skel[a].size());
                ++s->far_pairs;
            }
        }
        if (cnt == 0) s->min_rank = 0;
        s->mean_rank = cnt ? double(s->skel_total) / double(cnt) : 0.0;
        s->flops_s2n = s->flops_n2s;
        for (int64_t b = 0; b < st.n_leaves(); ++b) {
            const int64_t nb = st.node_size[st.leaf_node(b)];
            s->max_near = std::max<int64_t>(s->max_near, int64_t(st.near[b].size()));
            for (int64_t a : st.near[b]) {
                const int64_t na = st.node_size[st.leaf_node(a)];
                s->flops_l2l += 2.0 * double(nb) * double(na);
                s->near_entries += nb * na;
                ++s->near_pairs;
            }
        }
        s->ann_iterations = st.ann_iters;
        s->ann_recall = st.ann_recall;
        s->compress_seconds = st.compress_seconds;
    });
}

int gofmm_set_timing(gofmm_handle* h, int enable) {
    return guarded([&] {
        if (!h) gofmm::fail(GOFMM_ERR_ARG, "handle is NULL");
        if (enable < 0 || enable > 2) gofmm::fail(GOFMM_ERR_ARG, "timing level must be 0, 1 or 2");
        h->h.timing = enable;
    });
}

int gofmm_stage_times(gofmm_handle* h, float* ms, int n) {
    return guarded([&] {
        if (!h || !ms || n < 1) gofmm::fail(GOFMM_ERR_ARG, "bad arguments");
        gofmm::device_stage_times(h->h, ms, n);
    });
}

int64_t gofmm_view(const gofmm_handle* hd, int what, void* out) {
    if (!hd) return set_error(GOFMM_ERR_ARG, "handle is NULL");
    const gofmm::Structure& st = hd->h.st;
    auto csr = [&](const std::vector<std::vector<int64_t>>& lists) -> int64_t {
        int64_t total = int64_t(lists.size()) + 1;
        for (const auto& v : lists) total += int64_t(v.size());
        if (out) {
            int64_t* o = static_cast<int64_t*>(out);
            int64_t pos = 0;
            o[0] = 0;
            for (size_t i = 0; i < lists.size(); ++i) {
                pos += int64_t(lists[i].size());
                o[i + 1] = pos;
            }
            int64_t* vals = o + lists.size() + 1;
            for (const auto& v : lists) {
                std::memcpy(vals, v.data(), v.size() * sizeof(int64_t));
                vals += v.size();
            }
        }
        return total;
    };
    switch (what) {
        case 0:
            if (out) std::memcpy(out, st.perm.data(), st.perm.size() * sizeof(int64_t));
            return int64_t(st.perm.size());
        case 1: {
            const int64_t nl = st.n_leaves();
            if (out) {
                int64_t* o = static_cast<int64_t*>(out);
                for (int64_t b = 0; b < nl; ++b) o[b] = st.node_off[st.leaf_node(b)];
                o[nl] = st.n;
            }
            return nl + 1;
        }
        case 2: return csr(st.near);
        case 3: return csr(st.far);
        case 4: return csr(st.skel);
        case 5: {
            int64_t total = 0;
            for (const auto& v : st.P) total += int64_t(v.size());
            if (out) {
                double* o = static_cast<double*>(out);
                for (const auto& v : st.P) {
                    std::memcpy(o, v.data(), v.size() * sizeof(double));
                    o += v.size();
                }
            }
            return total;
        }
        default:
            return set_error(GOFMM_ERR_ARG, "unknown view");
    }
}

}  // extern "C"
