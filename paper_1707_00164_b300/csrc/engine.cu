// Batching and serving engine: many evaluations U_i = K~_i W_i in flight at
// once on one GPU, over any mix of resident compressed matrices and r.
//
// Every evaluation is the same sequence of stages as a single one (gather,
// then the tensor-core launches of its matrix's plan: N2S levels, S2S, S2N
// levels, leaf).  A step advances every admitted evaluation by one stage in
// ONE persistent grouped-GEMM launch whose tiles come from all of them (plus
// one gather launch per evaluation that starts), so uneven trees, ranks and
// right-hand-side counts are packed into the same kernel.  Evaluations
// arriving between steps join at the next step (continuous batching).  A
// task's arithmetic never depends on what else shares the launch (no
// split-K, fixed summation order), so a result is bitwise the same alone and
// in any mix.
//
// Admission is by memory: each evaluation needs its own right-hand-side
// workspace (tree-ordered W, skeleton weights and potentials in the RT
// layout), carved first-fit out of one pool allocated at creation; a request
// waits in FIFO order until its workspace fits.  A finished evaluation's
// workspace returns to the pool once the GPU has passed the step that
// completed it.
#include <algorithm>
#include <deque>
#include <memory>
#include <unordered_map>

#include "eval_tc.hpp"

namespace gofmm {

struct EngineRequest {
    int64_t id = 0;
    Handle* H = nullptr;
    TcPrec* T = nullptr;
    const float* W = nullptr;
    int64_t ldw = 0;
    float* U = nullptr;
    int64_t ldu = 0;
    int r = 0, n_rtiles = 0;
    int next = 0;  // 0: gather; 1 + k: launch k of the plan
    size_t ws_off = 0, ws_bytes = 0;
    uint8_t* rt_hi[3] = {nullptr, nullptr, nullptr};
    uint8_t* rt_lo[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t done_ev = nullptr;
};

struct Engine {
    int device = 0, precision = 0, mode = 0;
    int num_sms = 148;
    uint8_t* pool = nullptr;
    size_t pool_bytes = 0;
    std::map<size_t, size_t> free_blocks;  // offset -> size
    std::deque<EngineRequest*> queue;
    std::vector<EngineRequest*> active;
    std::vector<EngineRequest*> finishing;  // completed on the host side, waiting for their event
    std::unordered_map<int64_t, int> state;  // 0 queued, 1 running, 2 done
    int64_t next_id = 1;
    int* d_err = nullptr;
    int* h_err = nullptr;
    int* d_claims = nullptr;  // tile counters of one step's grouped launches (kClaimSlots)
    // statistics
    int64_t steps = 0, launches = 0, max_active = 0, completed = 0;
};

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool pool_alloc(Engine& E, size_t bytes, size_t& off) {
    for (auto it = E.free_blocks.begin(); it != E.free_blocks.end(); ++it) {
        if (it->second < bytes) continue;
        off = it->first;
        const size_t rest = it->second - bytes;
        E.free_blocks.erase(it);
        if (rest) E.free_blocks[off + bytes] = rest;
        return true;
    }
    return false;
}

void pool_free(Engine& E, size_t off, size_t bytes) {
    auto it = E.free_blocks.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != E.free_blocks.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        E.free_blocks.erase(nx);
    }
    if (it != E.free_blocks.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            E.free_blocks.erase(it);
        }
    }
}

size_t workspace_bytes(const TcPrec& T, int n_rtiles) {
    const size_t per = size_t(n_rtiles) * kTileBytes;
    const size_t chunks[3] = {size_t(T.wt_chunks), size_t(T.sk_chunks), size_t(T.sk_chunks)};
    size_t total = 0;
    for (size_t c : chunks) total += align_up(c * per, 256) * (T.split ? 2 : 1);
    return total;
}

void carve(EngineRequest& q, uint8_t* base) {
    const size_t per = size_t(q.n_rtiles) * kTileBytes;
    const size_t chunks[3] = {size_t(q.T->wt_chunks), size_t(q.T->sk_chunks), size_t(q.T->sk_chunks)};
    uint8_t* p = base + q.ws_off;
    for (int i = 0; i < 3; ++i) {
        q.rt_hi[i] = p;
        p += align_up(chunks[i] * per, 256);
        if (q.T->split) {
            q.rt_lo[i] = p;
            p += align_up(chunks[i] * per, 256);
        }
    }
}

// Requests whose final step the GPU has finished: release their workspace.
void retire(Engine& E) {
    for (size_t i = 0; i < E.finishing.size();) {
        EngineRequest* q = E.finishing[i];
        const cudaError_t e = cudaEventQuery(q->done_ev);
        if (e == cudaErrorNotReady) { ++i; continue; }
        if (e != cudaSuccess) fail(GOFMM_ERR_CUDA, std::string("engine event: ") + cudaGetErrorString(e));
        pool_free(E, q->ws_off, q->ws_bytes);
        cudaEventDestroy(q->done_ev);
        --q->H->inflight;
        E.state[q->id] = 2;
        ++E.completed;
        delete q;
        E.finishing[i] = E.finishing.back();
        E.finishing.pop_back();
    }
}

}  // namespace

Engine* engine_create(int device, int precision, int64_t pool_bytes) {
    if (precision != GOFMM_PREC_TF32 && precision != GOFMM_PREC_BF16 && precision != GOFMM_PREC_BF16X3)
        fail(GOFMM_ERR_UNSUPPORTED, "the engine runs the tensor-core precisions (TF32, BF16, BF16X3)");
    if (pool_bytes < (int64_t(1) << 20)) fail(GOFMM_ERR_ARG, "pool_bytes must be at least 1 MiB");
    DeviceGuard g(device);
    auto E = std::make_unique<Engine>();
    E->device = device;
    E->precision = precision;
    E->mode = mode_of(precision);
    CUDA_OK(cudaDeviceGetAttribute(&E->num_sms, cudaDevAttrMultiProcessorCount, device));
    E->pool_bytes = size_t(pool_bytes) / 256 * 256;
    E->pool = dalloc<uint8_t>(E->pool_bytes);
    E->free_blocks[0] = E->pool_bytes;
    E->d_err = dalloc<int>(1);
    E->d_claims = dalloc<int>(kClaimSlots);
    CUDA_OK(cudaMemset(E->d_err, 0, sizeof(int)));
    CUDA_OK(cudaMallocHost(&E->h_err, sizeof(int)));
    *E->h_err = 0;
    return E.release();
}

int64_t engine_submit(Engine& E, Handle& H, const float* W, int64_t ldw, float* U, int64_t ldu, int64_t r) {
    if (!W || !U) fail(GOFMM_ERR_ARG, "W and U must not be NULL");
    if (r < 1 || r > (int64_t(1) << 24) || ldw < r || ldu < r) fail(GOFMM_ERR_ARG, "need 1 <= r <= ld");
    if (H.st.prm.device != E.device) fail(GOFMM_ERR_ARG, "handle lives on another device than the engine");
    if (!H.dev || !H.dev->tc || !H.dev->tc->prec[E.mode])
        fail(GOFMM_ERR_ARG, "handle not prepared for the engine's precision: call gofmm_prepare first");
    auto q = std::make_unique<EngineRequest>();
    q->id = E.next_id++;
    q->H = &H;
    q->T = H.dev->tc->prec[E.mode];
    q->W = W;
    q->ldw = ldw;
    q->U = U;
    q->ldu = ldu;
    q->r = int(r);
    q->n_rtiles = int((r + 127) / 128);
    q->ws_bytes = workspace_bytes(*q->T, q->n_rtiles);
    if (q->ws_bytes > E.pool_bytes)
        fail(GOFMM_ERR_NOMEM, "request needs " + std::to_string(q->ws_bytes) + " bytes of workspace; the pool has " +
                                  std::to_string(E.pool_bytes));
    ++H.inflight;  // the plan may not be rebuilt until the request retires
    E.state[q->id] = 0;
    E.queue.push_back(q.release());
    return E.queue.back()->id;
}

int64_t engine_step(Engine& E, cudaStream_t s) {
    DeviceGuard g(E.device);
    if (*reinterpret_cast<volatile int*>(E.h_err) != 0)
        fail(GOFMM_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait (code " + std::to_string(*E.h_err) + ")");
    retire(E);
    // admission, first come first served, by workspace memory
    while (!E.queue.empty()) {
        EngineRequest* q = E.queue.front();
        size_t off = 0;
        if (!pool_alloc(E, q->ws_bytes, off)) break;
        q->ws_off = off;
        carve(*q, E.pool);
        q->next = 0;
        E.queue.pop_front();
        E.active.push_back(q);
        E.state[q->id] = 1;
    }
    if (E.active.empty()) return int64_t(E.queue.size() + E.finishing.size());
    E.max_active = std::max<int64_t>(E.max_active, int64_t(E.active.size()));

    // skip empty launches so every step does work for every request
    for (EngineRequest* q : E.active)
        while (q->next >= 1 && q->next <= int(q->T->launches.size()) && q->T->launches[q->next - 1].tasks.empty())
            ++q->next;

    // gathers of the requests that start now
    for (EngineRequest* q : E.active)
        if (q->next == 0) {
            launch_gather(E.mode, *q->T, q->W, q->ldw, q->H->dev->d_idx, q->rt_hi[0], q->rt_lo[0], q->r, s);
            ++E.launches;
        }

    // one grouped launch for everybody else (chunks of kMaxSegs requests)
    std::vector<EngineRequest*> gemm;
    for (EngineRequest* q : E.active)
        if (q->next >= 1 && q->next <= int(q->T->launches.size())) gemm.push_back(q);
    // the grouped launches claim their tiles from counters (whichever CTA is free)
    if (!gemm.empty()) CUDA_OK(cudaMemsetAsync(E.d_claims, 0, kClaimSlots * sizeof(int), s));
    for (size_t b0 = 0; b0 < gemm.size(); b0 += kMaxSegs) {
        const size_t nb = std::min<size_t>(kMaxSegs, gemm.size() - b0);
        // every segment brings the device tile list its plan keeps for its
        // launch and r (heaviest task first); the kernel maps a global tile
        // index to its segment, so a step uploads and sorts nothing
        TcParams p{};
        p.nsegs = int(nb);
        p.err = E.d_err;
        p.tiles = nullptr;
        int piece = 0, total = 0;
        bool gen = false;
        for (size_t k = 0; k < nb; ++k) {
            EngineRequest* q = gemm[b0 + k];
            TcLaunch& l = q->T->launches[q->next - 1];
            p.segs[k] = make_seg(*q->T, l, q->rt_hi, q->rt_lo, q->U, q->ldu, q->H->dev->d_idx, q->r);
            const auto tl = launch_tiles(l, q->n_rtiles, q->H->tc_order[E.mode]);
            p.segs[k].tiles = tl.first;
            p.segs[k].tile_base = total;
            total += tl.second;
            piece = std::max(piece, q->T->piece);
            gen = gen || q->T->gen;
        }
        p.ntiles = total;
        const size_t slot = b0 / kMaxSegs;
        p.tile_next = slot < size_t(kClaimSlots) ? E.d_claims + slot : nullptr;
        launch_gemm_mode(E.mode, piece, p, E.num_sms, s, gen);
        ++E.launches;
    }
    CUDA_OK(cudaMemcpyAsync(E.h_err, E.d_err, sizeof(int), cudaMemcpyDeviceToHost, s));

    // advance; requests past their last launch are complete once this step is
    std::vector<EngineRequest*> still;
    cudaEvent_t ev = nullptr;
    for (EngineRequest* q : E.active) {
        ++q->next;
        if (q->next > int(q->T->launches.size())) {
            if (!ev) {
                CUDA_OK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
                CUDA_OK(cudaEventRecord(ev, s));
                q->done_ev = ev;
            } else {
                CUDA_OK(cudaEventCreateWithFlags(&q->done_ev, cudaEventDisableTiming));
                CUDA_OK(cudaEventRecord(q->done_ev, s));
            }
            E.finishing.push_back(q);
        } else {
            still.push_back(q);
        }
    }
    E.active.swap(still);
    ++E.steps;
    return int64_t(E.queue.size() + E.active.size() + E.finishing.size());
}

int64_t engine_workspace(const Engine& E, Handle& H, int64_t r) {
    if (r < 1) fail(GOFMM_ERR_ARG, "r must be >= 1");
    if (!H.dev || !H.dev->tc || !H.dev->tc->prec[E.mode])
        fail(GOFMM_ERR_ARG, "handle not prepared for the engine's precision: call gofmm_prepare first");
    return int64_t(workspace_bytes(*H.dev->tc->prec[E.mode], int((r + 127) / 128)));
}

int engine_poll(Engine& E, int64_t id) {
    retire(E);
    auto it = E.state.find(id);
    if (it == E.state.end()) fail(GOFMM_ERR_ARG, "unknown request id");
    return it->second;
}

void engine_drain(Engine& E, cudaStream_t s) {
    DeviceGuard g(E.device);
    while (!E.queue.empty() || !E.active.empty()) {
        engine_step(E, s);
        // A step that leaves nothing running admitted nothing: the pool is
        // held by finished requests the GPU may still be completing.
        if (E.active.empty() && !E.queue.empty()) {
            if (E.finishing.empty())
                fail(GOFMM_ERR_NOMEM, "queued request does not fit the pool");  // cannot happen: submit checks
            CUDA_OK(cudaStreamSynchronize(s));
            retire(E);
        }
    }
    CUDA_OK(cudaStreamSynchronize(s));
    retire(E);
    if (*reinterpret_cast<volatile int*>(E.h_err) != 0)
        fail(GOFMM_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait (code " + std::to_string(*E.h_err) + ")");
}

void engine_stats(const Engine& E, int64_t* out, int n) {
    const int64_t v[7] = {E.steps, E.launches, E.max_active, E.completed, int64_t(E.queue.size()),
                          int64_t(E.active.size()), int64_t(E.finishing.size())};
    for (int i = 0; i < n && i < 7; ++i) out[i] = v[i];
}

void engine_destroy(Engine* E) {
    if (!E) return;
    int old = -1;
    cudaGetDevice(&old);
    cudaSetDevice(E->device);
    cudaDeviceSynchronize();
    for (EngineRequest* q : E->queue) {
        --q->H->inflight;
        delete q;
    }
    for (EngineRequest* q : E->active) {
        --q->H->inflight;
        delete q;
    }
    for (EngineRequest* q : E->finishing) {
        if (q->done_ev) cudaEventDestroy(q->done_ev);
        --q->H->inflight;
        delete q;
    }
    dfree(E->pool);
    dfree(E->d_err);
    dfree(E->d_claims);
    if (E->h_err) cudaFreeHost(E->h_err);
    delete E;
    if (old >= 0) cudaSetDevice(old);
}

}  // namespace gofmm

// ---------------------------------------------------------------------------
// Static batch: a fixed set of evaluations (matrix, r) whose merged step
// sequence is planned once (tile lists uploaded once, workspaces allocated
// once) and replayed; repeated calls with the same W/U pointers replay a
// CUDA graph of the whole sequence.
namespace gofmm {

struct BatchItem {
    Handle* H;
    TcPrec* T;
    int64_t epoch;  // the handle's plan epoch when the batch was made
    int r, n_rtiles;
    uint8_t* rt_hi[3];
    uint8_t* rt_lo[3];
};

struct BatchStep {
    std::vector<int> gathers;                   // items whose gather runs in this step
    struct Launch {
        std::vector<std::pair<int, int>> segs;  // (item, plan launch) per segment
        TcTile* d_tiles = nullptr;
        int ntiles = 0;
        int piece = 0;  // tallest task piece of the segments' plans
        bool gen = false;  // some segment generates its block tiles
    };
    std::vector<Launch> launches;
};

// Dependency-driven form: up to kMaxSegs items in one cooperative launch
// that runs every stage of all of them; each item's tiles in its own
// topological order, the items interleaved task by task.
struct BatchFused {
    std::vector<int> items;
    TcTile* d_tiles = nullptr;
    int ntiles = 0;
    int* d_counters = nullptr;          // the items' counters, then the tile counter
    std::vector<size_t> counter_off;    // per item
    size_t counter_ints = 0;
    int piece = 0;
    bool gen = false;
};

struct Batch {
    int device = 0, precision = 0, mode = 0, num_sms = 148;
    std::vector<BatchItem> items;
    std::vector<BatchStep> steps;
    bool fused = false;                 // every handle configured for the fused schedule
    std::vector<BatchFused> fused_launches;
    int* d_claims = nullptr;            // tile counters of the per-step launches (one each)
    int nclaims = 0;
    uint8_t* ws = nullptr;
    int* d_err = nullptr;
    int* h_err = nullptr;
    int launches_per_call = 0;
    cudaStream_t capture_stream = nullptr;
    std::map<std::vector<const void*>, std::pair<int, cudaGraphExec_t>> graphs;  // pointers -> (calls, graph)
};

Batch* batch_create(Handle* const* hs, const int64_t* r, int count, int precision) {
    if (count < 1) fail(GOFMM_ERR_ARG, "count must be >= 1");
    if (precision != GOFMM_PREC_TF32 && precision != GOFMM_PREC_BF16 && precision != GOFMM_PREC_BF16X3)
        fail(GOFMM_ERR_UNSUPPORTED, "batches run the tensor-core precisions (TF32, BF16, BF16X3)");
    auto B = std::make_unique<Batch>();
    B->precision = precision;
    B->mode = mode_of(precision);
    B->device = hs[0]->st.prm.device;
    DeviceGuard g(B->device);
    CUDA_OK(cudaDeviceGetAttribute(&B->num_sms, cudaDevAttrMultiProcessorCount, B->device));
    size_t total = 0;
    std::vector<size_t> sizes;
    for (int i = 0; i < count; ++i) {
        Handle& H = *hs[i];
        if (H.st.prm.device != B->device) fail(GOFMM_ERR_ARG, "all handles of a batch must live on one device");
        if (r[i] < 1 || r[i] > (int64_t(1) << 24)) fail(GOFMM_ERR_ARG, "r must be >= 1");
        if (!H.dev || !H.dev->tc || !H.dev->tc->prec[B->mode])
            fail(GOFMM_ERR_ARG, "handle not prepared for the batch precision: call gofmm_prepare first");
        BatchItem it{};
        it.H = &H;
        it.T = H.dev->tc->prec[B->mode];
        it.epoch = H.plan_epoch;
        it.r = int(r[i]);
        it.n_rtiles = int((r[i] + 127) / 128);
        B->items.push_back(it);
        sizes.push_back(workspace_bytes(*it.T, it.n_rtiles));
        total += sizes.back();
    }
    B->ws = dalloc<uint8_t>(total);
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
        EngineRequest q{};
        q.T = B->items[i].T;
        q.n_rtiles = B->items[i].n_rtiles;
        q.ws_off = off;
        carve(q, B->ws);
        for (int k = 0; k < 3; ++k) {
            B->items[i].rt_hi[k] = q.rt_hi[k];
            B->items[i].rt_lo[k] = q.rt_lo[k];
        }
        off += sizes[i];
    }
    B->fused = true;
    for (int i = 0; i < count; ++i) B->fused = B->fused && hs[i]->tc_schedule[B->mode] == GOFMM_SCHED_FUSED;
    if (B->fused) {
        for (int c0 = 0; c0 < count; c0 += kMaxSegs) {
            BatchFused bf;
            const int c1 = std::min(count, c0 + kMaxSegs);
            size_t off = 0;
            std::vector<const std::vector<int32_t>*> orders;
            for (int i = c0; i < c1; ++i) {
                const BatchItem& it = B->items[i];
                const TcFused& F = it.T->fused;
                bf.items.push_back(i);
                bf.counter_off.push_back(off);
                off += size_t(F.ncounters) * size_t(it.n_rtiles);
                bf.piece = std::max(bf.piece, it.T->piece);
                bf.gen = bf.gen || it.T->gen;
                orders.push_back(&fused_order(F, it.H->tc_order[B->mode]));
            }
            bf.counter_ints = off + 1;  // + the tile counter
            bf.d_counters = dalloc<int>(bf.counter_ints);
            // interleave the items task by task; each keeps its own order
            std::vector<TcTile> tiles;
            std::vector<size_t> pos(orders.size(), 0);
            for (bool more = true; more;) {
                more = false;
                for (size_t k = 0; k < orders.size(); ++k) {
                    if (pos[k] >= orders[k]->size()) continue;
                    more = true;
                    const int32_t task = (*orders[k])[pos[k]++];
                    const BatchItem& it = B->items[bf.items[k]];
                    task_tiles(tiles, int32_t(k), task, it.T->fused.tasks[size_t(task)], it.n_rtiles);
                }
            }
            bf.d_tiles = dupload(tiles);
            bf.ntiles = int(tiles.size());
            B->launches_per_call += (c1 - c0) + 1;  // gathers + one GEMM launch
            B->fused_launches.push_back(std::move(bf));
        }
    }
    // the step sequence: every item advances one stage per step
    std::vector<int> next(count, 0);
    for (;;) {
        BatchStep st;
        std::vector<int> gemm;
        for (int i = 0; i < count; ++i) {
            const auto& L = B->items[i].T->launches;
            while (next[i] >= 1 && next[i] <= int(L.size()) && L[next[i] - 1].tasks.empty()) ++next[i];
            if (next[i] == 0) st.gathers.push_back(i);
            else if (next[i] <= int(L.size())) gemm.push_back(i);
        }
        if (st.gathers.empty() && gemm.empty()) break;
        for (size_t b0 = 0; b0 < gemm.size(); b0 += kMaxSegs) {
            BatchStep::Launch bl;
            std::vector<std::pair<int64_t, TcTile>> tiles;
            for (size_t k = 0; b0 + k < gemm.size() && k < size_t(kMaxSegs); ++k) {
                const int i = gemm[b0 + k];
                const TcLaunch& l = B->items[i].T->launches[next[i] - 1];
                bl.segs.emplace_back(i, next[i] - 1);
                bl.piece = std::max(bl.piece, B->items[i].T->piece);
                bl.gen = bl.gen || B->items[i].T->gen;
                for (size_t t = 0; t < l.tasks.size(); ++t) {
                    std::vector<TcTile> tt;
                    task_tiles(tt, int32_t(k), int32_t(t), l.tasks[t], B->items[i].n_rtiles);
                    for (const TcTile& x : tt)
                        tiles.emplace_back(int64_t(l.tasks[t].nchunks) * l.tasks[t].n_pad * x.pad + 1, x);
                }
            }
            std::stable_sort(tiles.begin(), tiles.end(),
                             [](const std::pair<int64_t, TcTile>& a, const std::pair<int64_t, TcTile>& b) {
                                 return a.first > b.first;
                             });
            std::vector<TcTile> tv;
            for (auto& t : tiles) tv.push_back(t.second);
            bl.d_tiles = dupload(tv);
            bl.ntiles = int(tv.size());
            st.launches.push_back(std::move(bl));
        }
        for (int i : st.gathers) next[i] = 1;
        for (int i : gemm) ++next[i];
        if (!B->fused) B->launches_per_call += int(st.gathers.size() + st.launches.size());
        B->steps.push_back(std::move(st));
    }
    B->d_err = dalloc<int>(1);
    for (const BatchStep& st : B->steps) B->nclaims += int(st.launches.size());
    B->d_claims = dalloc<int>(size_t(std::max(1, B->nclaims)));
    CUDA_OK(cudaMemset(B->d_err, 0, sizeof(int)));
    CUDA_OK(cudaMallocHost(&B->h_err, sizeof(int)));
    *B->h_err = 0;
    CUDA_OK(cudaStreamCreateWithFlags(&B->capture_stream, cudaStreamNonBlocking));
    return B.release();
}

static void batch_launch(Batch& B, const float* const* W, const int64_t* ldw, float* const* U, const int64_t* ldu,
                         cudaStream_t s) {
    if (B.fused) {
        for (const BatchFused& bf : B.fused_launches) {
            TcParams p{};
            p.nsegs = int(bf.items.size());
            p.err = B.d_err;
            p.tiles = bf.d_tiles;
            p.ntiles = bf.ntiles;
            for (size_t k = 0; k < bf.items.size(); ++k) {
                const int i = bf.items[k];
                const BatchItem& it = B.items[i];
                launch_gather(B.mode, *it.T, W[i], ldw[i], it.H->dev->d_idx, it.rt_hi[0], it.rt_lo[0], it.r, s);
                const TcFused& F = it.T->fused;
                TcSeg g = make_seg(*it.T, it.T->launches.front(), it.rt_hi, it.rt_lo, U[i], ldu[i],
                                   it.H->dev->d_idx, it.r);
                g.tasks = F.d_tasks;
                g.slabs = F.d_slabs;
                g.dep_off = F.d_dep_off;
                g.deps = F.d_deps;
                g.sig = F.d_sig;
                g.counters = bf.d_counters + bf.counter_off[k];
                g.dep_nrt = it.n_rtiles;
                p.segs[k] = g;
            }
            CUDA_OK(cudaMemsetAsync(bf.d_counters, 0, bf.counter_ints * sizeof(int), s));
            p.tile_next = bf.d_counters + (bf.counter_ints - 1);
            launch_gemm_coop_mode(B.mode, bf.piece, p, B.num_sms, s, bf.gen);
        }
        CUDA_OK(cudaMemcpyAsync(B.h_err, B.d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        return;
    }
    // the per-step launches claim their tiles from counters
    if (B.nclaims > 0) CUDA_OK(cudaMemsetAsync(B.d_claims, 0, size_t(B.nclaims) * sizeof(int), s));
    int claim = 0;
    for (const BatchStep& st : B.steps) {
        for (int i : st.gathers) {
            const BatchItem& it = B.items[i];
            launch_gather(B.mode, *it.T, W[i], ldw[i], it.H->dev->d_idx, it.rt_hi[0], it.rt_lo[0], it.r, s);
        }
        for (const BatchStep::Launch& bl : st.launches) {
            TcParams p{};
            p.nsegs = int(bl.segs.size());
            p.err = B.d_err;
            p.tiles = bl.d_tiles;
            p.ntiles = bl.ntiles;
            for (size_t k = 0; k < bl.segs.size(); ++k) {
                const int i = bl.segs[k].first;
                const BatchItem& it = B.items[i];
                p.segs[k] = make_seg(*it.T, it.T->launches[bl.segs[k].second], it.rt_hi, it.rt_lo, U[i], ldu[i],
                                     it.H->dev->d_idx, it.r);
            }
            p.tile_next = B.d_claims + claim++;
            launch_gemm_mode(B.mode, bl.piece, p, B.num_sms, s, bl.gen);
        }
    }
    CUDA_OK(cudaMemcpyAsync(B.h_err, B.d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
}

int batch_evaluate(Batch& B, const float* const* W, const int64_t* ldw, float* const* U, const int64_t* ldu,
                   cudaStream_t s) {
    DeviceGuard g(B.device);
    if (*reinterpret_cast<volatile int*>(B.h_err) != 0)
        fail(GOFMM_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait (code " + std::to_string(*B.h_err) + ")");
    std::vector<const void*> key;
    for (size_t i = 0; i < B.items.size(); ++i) {
        if (B.items[i].H->plan_epoch != B.items[i].epoch)
            fail(GOFMM_ERR_ARG, "the plan of batch item " + std::to_string(i) +
                                    " was rebuilt after the batch was created: create the batch again");
        if (!W[i] || !U[i] || ldw[i] < B.items[i].r || ldu[i] < B.items[i].r)
            fail(GOFMM_ERR_ARG, "bad W/U of batch item " + std::to_string(i));
        key.push_back(W[i]);
        key.push_back(U[i]);
        key.push_back(reinterpret_cast<const void*>(ldw[i]));
        key.push_back(reinterpret_cast<const void*>(ldu[i]));
    }
    auto& e = B.graphs[key];
    ++e.first;
    if (!e.second && e.first >= 2) {
        cudaGraph_t gr = nullptr;
        CUDA_OK(cudaStreamBeginCapture(B.capture_stream, cudaStreamCaptureModeThreadLocal));
        try {
            batch_launch(B, W, ldw, U, ldu, B.capture_stream);
        } catch (...) {
            cudaStreamEndCapture(B.capture_stream, &gr);
            if (gr) cudaGraphDestroy(gr);
            throw;
        }
        CUDA_OK(cudaStreamEndCapture(B.capture_stream, &gr));
        const cudaError_t ie = cudaGraphInstantiate(&e.second, gr, 0);
        cudaGraphDestroy(gr);
        CUDA_OK(ie);
    }
    if (e.second) CUDA_OK(cudaGraphLaunch(e.second, s));
    else batch_launch(B, W, ldw, U, ldu, s);
    return B.launches_per_call;
}

int batch_error(const Batch& B) { return *B.h_err; }

void batch_destroy(Batch* B) {
    if (!B) return;
    int old = -1;
    cudaGetDevice(&old);
    cudaSetDevice(B->device);
    cudaDeviceSynchronize();
    for (auto& kv : B->graphs)
        if (kv.second.second) cudaGraphExecDestroy(kv.second.second);
    for (BatchStep& st : B->steps)
        for (auto& bl : st.launches) dfree(bl.d_tiles);
    for (BatchFused& bf : B->fused_launches) {
        dfree(bf.d_tiles);
        dfree(bf.d_counters);
    }
    dfree(B->ws);
    dfree(B->d_err);
    dfree(B->d_claims);
    if (B->h_err) cudaFreeHost(B->h_err);
    if (B->capture_stream) cudaStreamDestroy(B->capture_stream);
    delete B;
    if (old >= 0) cudaSetDevice(old);
}

}  // namespace gofmm
