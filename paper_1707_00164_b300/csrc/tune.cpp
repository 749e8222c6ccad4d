// Autotuner of the tensor-core launch configuration (task piece height,
// schedule, fused tile order) and its JSON cache file.
//
// A configuration changes how the grouped GEMMs are cut into tiles and in
// which order the tiles run, never a task's summation order, so every
// candidate computes bitwise the same U and the tuner may pick on speed
// alone.  Candidates are timed with CUDA events on the caller's stream on
// scratch right-hand sides; the choice is stored under a key made of the
// compressed structure(s), the number of 128-column tiles of r, the
// precision and the GPU, so a later run on the same problem reads it back
// without measuring.
#include <cuda_runtime.h>
#include <unistd.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <memory>
#include <sstream>
#include <string>
#include <utility>
#include <vector>

#include "eval_state.hpp"
#include "gofmm_internal.hpp"

namespace gofmm {
namespace {

// ------------------------------------------------------------------ key --
struct Fnv1a {
    uint64_t h = 1469598103934665603ull;
    void bytes(const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    }
    template <class T>
    void val(const T& x) {
        bytes(&x, sizeof x);
    }
};

void hash_structure(Fnv1a& f, const Structure& st) {
    f.val(st.n);
    f.val(st.depth);
    f.val(st.prm.cache_mode);
    for (int64_t x : st.node_size) f.val(x);
    for (const auto& s : st.skel) f.val(int64_t(s.size()));
    for (const auto& l : st.near) {
        f.val(int64_t(l.size()));
        for (int64_t x : l) f.val(x);
    }
    for (const auto& l : st.far) {
        f.val(int64_t(l.size()));
        for (int64_t x : l) f.val(x);
    }
}

std::string device_tag(int device) {
    cudaDeviceProp p{};
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) {
        cudaGetLastError();
        return "no-gpu";
    }
    return std::string(p.name) + "/" + std::to_string(p.multiProcessorCount);
}

bool tensor_precision(int precision) {
    return precision == GOFMM_PREC_TF32 || precision == GOFMM_PREC_BF16 || precision == GOFMM_PREC_BF16X3;
}

// ----------------------------------------------------------------- JSON --
// Just enough JSON for the cache file: objects, arrays, strings (with the
// two-character escapes), numbers, true/false/null.
struct JVal {
    enum Kind { NUL, BOOL, NUM, STR, ARR, OBJ } kind = NUL;
    double num = 0;
    std::string str;
    std::vector<JVal> arr;
    std::vector<std::pair<std::string, JVal>> obj;

    const JVal* get(const std::string& k) const {
        for (const auto& kv : obj)
            if (kv.first == k) return &kv.second;
        return nullptr;
    }
    static JVal number(double x) {
        JVal v;
        v.kind = NUM;
        v.num = x;
        return v;
    }
    static JVal string(const std::string& s) {
        JVal v;
        v.kind = STR;
        v.str = s;
        return v;
    }
};

struct JParser {
    const std::string& s;
    size_t i = 0;
    explicit JParser(const std::string& text) : s(text) {}

    [[noreturn]] void bad(const char* what) const {
        fail(GOFMM_ERR_ARG, std::string("autotune cache: ") + what + " at byte " + std::to_string(i));
    }
    void ws() {
        while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t')) ++i;
    }
    bool lit(const char* w) {
        const size_t n = std::strlen(w);
        if (s.compare(i, n, w) != 0) return false;
        i += n;
        return true;
    }
    std::string str() {
        if (i >= s.size() || s[i] != '"') bad("string expected");
        ++i;
        std::string out;
        while (i < s.size() && s[i] != '"') {
            char c = s[i++];
            if (c == '\\') {
                if (i >= s.size()) bad("bad escape");
                const char e = s[i++];
                c = e == 'n' ? '\n' : e == 't' ? '\t' : e == 'r' ? '\r' : e;
                if (e != '"' && e != '\\' && e != '/' && e != 'n' && e != 't' && e != 'r') bad("unsupported escape");
            }
            out.push_back(c);
        }
        if (i >= s.size()) bad("unterminated string");
        ++i;
        return out;
    }
    JVal value(int depth = 0) {
        if (depth > 32) bad("nesting too deep");
        ws();
        if (i >= s.size()) bad("value expected");
        JVal v;
        const char c = s[i];
        if (c == '{') {
            v.kind = JVal::OBJ;
            ++i;
            ws();
            if (i < s.size() && s[i] == '}') { ++i; return v; }
            for (;;) {
                ws();
                std::string k = str();
                ws();
                if (i >= s.size() || s[i] != ':') bad("':' expected");
                ++i;
                v.obj.emplace_back(std::move(k), value(depth + 1));
                ws();
                if (i < s.size() && s[i] == ',') { ++i; continue; }
                if (i < s.size() && s[i] == '}') { ++i; return v; }
                bad("',' or '}' expected");
            }
        }
        if (c == '[') {
            v.kind = JVal::ARR;
            ++i;
            ws();
            if (i < s.size() && s[i] == ']') { ++i; return v; }
            for (;;) {
                v.arr.push_back(value(depth + 1));
                ws();
                if (i < s.size() && s[i] == ',') { ++i; continue; }
                if (i < s.size() && s[i] == ']') { ++i; return v; }
                bad("',' or ']' expected");
            }
        }
        if (c == '"') return JVal::string(str());
        if (lit("true")) { v.kind = JVal::BOOL; v.num = 1; return v; }
        if (lit("false")) { v.kind = JVal::BOOL; return v; }
        if (lit("null")) return v;
        const char* b = s.c_str() + i;
        char* e = nullptr;
        const double x = std::strtod(b, &e);
        if (e == b) bad("value expected");
        i += size_t(e - b);
        return JVal::number(x);
    }
};

void emit(std::ostringstream& o, const JVal& v) {
    switch (v.kind) {
        case JVal::NUL: o << "null"; break;
        case JVal::BOOL: o << (v.num != 0 ? "true" : "false"); break;
        case JVal::NUM: {
            char buf[40];
            std::snprintf(buf, sizeof buf, "%.17g", v.num);
            o << buf;
            break;
        }
        case JVal::STR: {
            o << '"';
            for (char c : v.str) {
                if (c == '"' || c == '\\') o << '\\' << c;
                else if (c == '\n') o << "\\n";
                else o << c;
            }
            o << '"';
            break;
        }
        case JVal::ARR: {
            o << '[';
            for (size_t k = 0; k < v.arr.size(); ++k) {
                if (k) o << ", ";
                emit(o, v.arr[k]);
            }
            o << ']';
            break;
        }
        case JVal::OBJ: {
            o << '{';
            for (size_t k = 0; k < v.obj.size(); ++k) {
                if (k) o << ", ";
                emit(o, JVal::string(v.obj[k].first));
                o << ": ";
                emit(o, v.obj[k].second);
            }
            o << '}';
            break;
        }
    }
}

constexpr const char* kFormat = "gofmm-autotune";

// Entries of the cache file (empty if the file does not exist).
std::vector<JVal> load_cache(const char* path) {
    std::ifstream f(path, std::ios::binary);
    if (!f) return {};
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string text = ss.str();
    JParser p(text);
    JVal root = p.value();
    p.ws();
    if (p.i != text.size()) p.bad("trailing characters");
    const JVal* fmt = root.get("format");
    const JVal* ent = root.get("entries");
    if (root.kind != JVal::OBJ || !fmt || fmt->kind != JVal::STR || fmt->str != kFormat || !ent ||
        ent->kind != JVal::ARR)
        fail(GOFMM_ERR_ARG, std::string("not a gofmm autotune cache: ") + path);
    return ent->arr;
}

void store_cache(const char* path, const std::vector<JVal>& entries) {
    std::ostringstream o;
    o << "{\"format\": \"" << kFormat << "\", \"version\": 1, \"entries\": [\n";
    for (size_t k = 0; k < entries.size(); ++k) {
        o << "  ";
        emit(o, entries[k]);
        o << (k + 1 < entries.size() ? ",\n" : "\n");
    }
    o << "]}\n";
    const std::string tmp = std::string(path) + ".tmp" + std::to_string(::getpid());
    {
        std::ofstream f(tmp, std::ios::binary | std::ios::trunc);
        if (!f) fail(GOFMM_ERR_ARG, std::string("cannot write the autotune cache: ") + tmp);
        f << o.str();
        if (!f) fail(GOFMM_ERR_ARG, std::string("cannot write the autotune cache: ") + tmp);
    }
    if (std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        fail(GOFMM_ERR_ARG, std::string("cannot replace the autotune cache: ") + path);
    }
}

const JVal* find_entry(const std::vector<JVal>& entries, const std::string& key) {
    for (const JVal& e : entries) {
        const JVal* k = e.get("key");
        if (e.kind == JVal::OBJ && k && k->kind == JVal::STR && k->str == key) return &e;
    }
    return nullptr;
}

int num_field(const JVal& e, const char* name) {
    const JVal* v = e.get(name);
    if (!v || v->kind != JVal::NUM) fail(GOFMM_ERR_ARG, std::string("autotune cache entry without ") + name);
    return int(v->num);
}

JVal make_entry(const TuneResult& t, int precision, int64_t r, int count, const std::string& dev) {
    JVal e;
    e.kind = JVal::OBJ;
    e.obj.emplace_back("key", JVal::string(t.key));
    e.obj.emplace_back("device", JVal::string(dev));
    e.obj.emplace_back("precision", JVal::number(precision));
    e.obj.emplace_back("r_tiles", JVal::number(double((r + 127) / 128)));
    e.obj.emplace_back("instances", JVal::number(count));
    e.obj.emplace_back("piece", JVal::number(t.piece));
    e.obj.emplace_back("schedule", JVal::number(t.schedule));
    e.obj.emplace_back("order", JVal::number(t.order));
    JVal c;
    c.kind = JVal::ARR;
    for (int k = 0; k < t.n; ++k) {
        JVal x;
        x.kind = JVal::OBJ;
        x.obj.emplace_back("piece", JVal::number(t.cand_piece[k]));
        x.obj.emplace_back("schedule", JVal::number(t.cand_schedule[k]));
        x.obj.emplace_back("order", JVal::number(t.cand_order[k]));
        x.obj.emplace_back("ms", JVal::number(t.cand_ms[k]));
        c.arr.push_back(std::move(x));
    }
    e.obj.emplace_back("candidates", std::move(c));
    return e;
}

// Cache lookup shared by both tuners: true (and *out filled) on a hit.
bool cached_choice(const char* path, const std::string& key, TuneResult& out) {
    if (!path) return false;
    const std::vector<JVal> entries = load_cache(path);
    const JVal* e = find_entry(entries, key);
    if (!e) return false;
    out.piece = num_field(*e, "piece");
    out.schedule = num_field(*e, "schedule");
    out.order = num_field(*e, "order");
    out.from_cache = 1;
    out.n = 0;
    return true;
}

void remember(const char* path, const TuneResult& t, int precision, int64_t r, int count, const std::string& dev) {
    if (!path) return;
    std::vector<JVal> entries = load_cache(path);  // re-read: another process may have added entries
    JVal e = make_entry(t, precision, r, count, dev);
    bool replaced = false;
    for (JVal& x : entries) {
        const JVal* k = x.get("key");
        if (k && k->kind == JVal::STR && k->str == t.key) {
            x = e;
            replaced = true;
        }
    }
    if (!replaced) entries.push_back(std::move(e));
    store_cache(path, entries);
}

// Median of the CUDA-event time of `reps` calls of f after `warm` untimed ones.
template <class F>
float time_median(F&& f, cudaStream_t s, int warm, int reps) {
    for (int k = 0; k < warm; ++k) f();
    std::vector<cudaEvent_t> ev(size_t(reps) + 1);
    for (auto& e : ev) CUDA_OK(cudaEventCreate(&e));
    std::vector<float> ms(size_t(reps), 0.f);
    try {
        CUDA_OK(cudaEventRecord(ev[0], s));
        for (int k = 0; k < reps; ++k) {
            f();
            CUDA_OK(cudaEventRecord(ev[size_t(k) + 1], s));
        }
        CUDA_OK(cudaEventSynchronize(ev[size_t(reps)]));
        for (int k = 0; k < reps; ++k) CUDA_OK(cudaEventElapsedTime(&ms[size_t(k)], ev[size_t(k)], ev[size_t(k) + 1]));
    } catch (...) {
        for (auto& e : ev) cudaEventDestroy(e);
        throw;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
}

// Device scratch freed on every exit path.  Right-hand sides are filled
// with pseudo-random values in [-1, 1) (a 64-bit xorshift): on all-zero
// operands the same launches ran 3-5 % faster (split BF16x3), which is not
// the time a caller's data takes.
struct DevBuf {
    void* p = nullptr;
    explicit DevBuf(size_t bytes, bool random = false) {
        const cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(e == cudaErrorMemoryAllocation ? GOFMM_ERR_NOMEM : GOFMM_ERR_CUDA,
                 std::string("autotune scratch: ") + cudaGetErrorString(e));
        }
        if (!random) {
            CUDA_OK(cudaMemset(p, 0, bytes));
            return;
        }
        std::vector<float> h(bytes / sizeof(float));
        uint64_t x = 0x9E3779B97F4A7C15ull;
        for (float& v : h) {
            x ^= x << 13;
            x ^= x >> 7;
            x ^= x << 17;
            v = float(int64_t(x >> 40) - (int64_t(1) << 23)) * (1.0f / float(1 << 23));
        }
        CUDA_OK(cudaMemcpy(p, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
};

constexpr int kWarm = 3, kReps = 7;

}  // namespace

std::string tune_key_batch(Handle* const* hs, const int64_t* r, int count, int precision) {
    if (count < 1 || !hs) fail(GOFMM_ERR_ARG, "need at least one handle");
    Fnv1a f;
    f.val(precision);
    f.val(count);
    for (int i = 0; i < count; ++i) {
        if (!hs[i]) fail(GOFMM_ERR_ARG, "NULL handle");
        if (r[i] < 1) fail(GOFMM_ERR_ARG, "r must be >= 1");
        hash_structure(f, hs[i]->st);
        f.val(int64_t((r[i] + 127) / 128));
    }
    const std::string dev = device_tag(hs[0]->st.prm.device);
    f.bytes(dev.data(), dev.size());
    char buf[32];
    std::snprintf(buf, sizeof buf, "%c%016llx", count == 1 ? 'e' : 'b', static_cast<unsigned long long>(f.h));
    return buf;
}

std::string tune_key(const Handle& H, int64_t r, int precision) {
    Handle* h = const_cast<Handle*>(&H);
    return tune_key_batch(&h, &r, 1, precision);
}

TuneResult autotune(Handle& H, int64_t r, int precision, const char* cache_path, void* stream) {
    if (!tensor_precision(precision)) fail(GOFMM_ERR_ARG, "autotuning is for the tensor-core precisions");
    if (r < 1 || r > (int64_t(1) << 24)) fail(GOFMM_ERR_ARG, "r must be >= 1");
    TuneResult res;
    res.key = tune_key(H, r, precision);
    if (cached_choice(cache_path, res.key, res)) {
        device_set_tc_config(H, precision, res.piece, res.schedule, res.order);
        return res;
    }
    DeviceGuard g(H.st.prm.device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    device_prepare(H, r, precision);
    const int64_t n = H.st.n;
    DevBuf W(size_t(n) * size_t(r) * sizeof(float), true), U(size_t(n) * size_t(r) * sizeof(float));
    const int saved_timing = H.timing;
    H.timing = 0;  // the production path, graph replay included
    // the per-stage schedules take the heap order (their critical-path
    // order never won); the single dependency-driven launch every order, the
    // hybrid the critical-path and locality orders
    const int cands[8][2] = {{GOFMM_SCHED_FUSED, GOFMM_ORDER_CRITICAL},  {GOFMM_SCHED_FUSED, GOFMM_ORDER_LOCAL},
                             {GOFMM_SCHED_FUSED, GOFMM_ORDER_LEVELS},    {GOFMM_SCHED_FUSED, GOFMM_ORDER_READY},
                             {GOFMM_SCHED_STAGED, GOFMM_ORDER_LOCAL},    {GOFMM_SCHED_PAIR, GOFMM_ORDER_LOCAL},
                             {GOFMM_SCHED_HYBRID, GOFMM_ORDER_CRITICAL}, {GOFMM_SCHED_HYBRID, GOFMM_ORDER_LOCAL}};
    float best = 0.f;
    const bool gen_plan = H.st.prm.cache_mode == GOFMM_CACHE_NONE;  // blocks generated in the kernel
    try {
        for (int piece : {256, 128})
            for (const auto& c : cands) {
                if (gen_plan && c[0] == GOFMM_SCHED_PAIR) continue;  // the pair kernel reads cached blocks
                device_set_tc_config(H, precision, piece, c[0], c[1]);
                device_prepare(H, r, precision);
                const float ms = time_median(
                    [&] { device_evaluate(H, W.p, r, U.p, r, r, GOFMM_DTYPE_F32, precision, s, 0); }, s, kWarm,
                    kReps);
                device_synchronize(H, s);  // a kernel that gave up a wait fails the tuning
                res.cand_piece[res.n] = piece;
                res.cand_schedule[res.n] = c[0];
                res.cand_order[res.n] = c[1];
                res.cand_ms[res.n] = ms;
                if (res.n == 0 || ms < best) {
                    best = ms;
                    res.piece = piece;
                    res.schedule = c[0];
                    res.order = c[1];
                }
                ++res.n;
            }
    } catch (...) {
        H.timing = saved_timing;
        throw;
    }
    H.timing = saved_timing;
    device_set_tc_config(H, precision, res.piece, res.schedule, res.order);
    device_prepare(H, r, precision);
    remember(cache_path, res, precision, r, 1, device_tag(H.st.prm.device));
    return res;
}

TuneResult autotune_batch(Handle* const* hs, const int64_t* r, int count, int precision, const char* cache_path,
                          void* stream) {
    if (!tensor_precision(precision)) fail(GOFMM_ERR_ARG, "autotuning is for the tensor-core precisions");
    TuneResult res;
    res.key = tune_key_batch(hs, r, count, precision);
    // a batch runs either as one dependency-driven launch per 64 items (every
    // handle on the fused schedule) or as one launch per stage step
    auto apply = [&](int piece, int schedule, int order) {
        for (int i = 0; i < count; ++i) device_set_tc_config(*hs[i], precision, piece, schedule, order);
    };
    if (cached_choice(cache_path, res.key, res)) {
        apply(res.piece, res.schedule, res.order);
        return res;
    }
    DeviceGuard g(hs[0]->st.prm.device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<std::unique_ptr<DevBuf>> bufs;
    std::vector<const float*> W(size_t(count), nullptr);
    std::vector<float*> U(size_t(count), nullptr);
    std::vector<int64_t> ld(r, r + count);
    for (int i = 0; i < count; ++i) {
        bufs.push_back(std::make_unique<DevBuf>(size_t(hs[i]->st.n) * size_t(r[i]) * sizeof(float), true));
        W[size_t(i)] = static_cast<const float*>(bufs.back()->p);
        bufs.push_back(std::make_unique<DevBuf>(size_t(hs[i]->st.n) * size_t(r[i]) * sizeof(float)));
        U[size_t(i)] = static_cast<float*>(bufs.back()->p);
    }
    float best = 0.f;
    static const int cands[4][2] = {{256, GOFMM_SCHED_FUSED}, {256, GOFMM_SCHED_STAGED},
                                    {128, GOFMM_SCHED_FUSED}, {128, GOFMM_SCHED_STAGED}};
    for (const auto& c : cands) {
        const int piece = c[0], schedule = c[1];
        apply(piece, schedule, GOFMM_ORDER_LOCAL);
        for (int i = 0; i < count; ++i) device_prepare(*hs[i], r[i], precision);
        Batch* B = batch_create(hs, r, count, precision);
        float ms = 0.f;
        try {
            ms = time_median([&] { batch_evaluate(*B, W.data(), ld.data(), U.data(), ld.data(), s); }, s, kWarm,
                             kReps);
            if (const int e = batch_error(*B))
                fail(GOFMM_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait (code " + std::to_string(e) + ")");
        } catch (...) {
            batch_destroy(B);
            throw;
        }
        batch_destroy(B);
        res.cand_piece[res.n] = piece;
        res.cand_schedule[res.n] = schedule;
        res.cand_order[res.n] = GOFMM_ORDER_LOCAL;
        res.cand_ms[res.n] = ms;
        if (res.n == 0 || ms < best) {
            best = ms;
            res.piece = piece;
            res.schedule = schedule;
            res.order = GOFMM_ORDER_LOCAL;
        }
        ++res.n;
    }
    apply(res.piece, res.schedule, res.order);
    for (int i = 0; i < count; ++i) device_prepare(*hs[i], r[i], precision);
    remember(cache_path, res, precision, r[0], count, device_tag(hs[0]->st.prm.device));
    return res;
}

}  // namespace gofmm
