// Device-side state of one compressed matrix: the evaluation plan, the
// cached K blocks and interpolation matrices in every element type used,
// and the evaluation workspace.  Shared by the SIMT path (eval.cu) and the
// tensor-core path (eval_tc.cu).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <tuple>
#include <string>
#include <utility>
#include <vector>

#include "eval_plan.hpp"
#include "gofmm_internal.hpp"

namespace gofmm {

#define CUDA_OK(x)                                                                                   \
    do {                                                                                             \
        cudaError_t e_ = (x);                                                                        \
        if (e_ != cudaSuccess) fail(GOFMM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)


struct DeviceGuard {
    int old = -1;
    explicit DeviceGuard(int dev) {
        CUDA_OK(cudaGetDevice(&old));
        if (old != dev) CUDA_OK(cudaSetDevice(dev));
    }
    ~DeviceGuard() {
        int cur = -1;
        if (old >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != old) cudaSetDevice(old);
    }
};

template <class T>
inline T* dalloc(size_t n) {
    if (n == 0) return nullptr;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? GOFMM_ERR_NOMEM : GOFMM_ERR_CUDA,
             std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return static_cast<T*>(p);
}
template <class T>
inline T* dupload(const std::vector<T>& v) {
    T* p = dalloc<T>(v.size());
    if (p) CUDA_OK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}
inline void dfree(void* p) {
    if (p) cudaFree(p);
}


// ---------------------------------------------------------------- plan --
struct Launch {
    int stage = 0;
    std::vector<Task> tasks;
    std::vector<Slab> slabs;
    Task* d_tasks = nullptr;
    Slab* d_slabs = nullptr;
    std::map<int, std::pair<Tile*, int>> tiles;  // tile height -> (device tiles, count)
};

struct Family {  // stores and workspace of one element type
    void* kstore = nullptr;
    void* pstore = nullptr;
    bool stores = false;
    int64_t ws_r = 0;
    void* WT = nullptr;
    void* WTIL = nullptr;
    void* UTIL = nullptr;
    // device staging of the host-buffer entry points: slot 0 (synchronous
    // calls) and, for asynchronous calls, which take the slots in turn, all
    // kStageSlots: the copy in of one call, the evaluation of the one before
    // and the copy out of the one before that run at once.  slot_free[k] is
    // recorded when the copy out of slot k's last call is done.
    static constexpr int kStageSlots = 3;
    void* sW[kStageSlots] = {nullptr, nullptr, nullptr};
    void* sU[kStageSlots] = {nullptr, nullptr, nullptr};
    int64_t stage_r = 0;
    int stage_next = 0;
    cudaEvent_t slot_free[kStageSlots] = {nullptr, nullptr, nullptr};
};

struct DeviceState {
    int device = 0;
    int64_t n = 0, S_tot = 0;
    std::vector<int64_t> skel_off, p_off, pt_off;
    std::vector<int64_t> idx;  // perm, then packed skeletons
    int64_t* d_idx = nullptr;
    double* d_pts64 = nullptr;
    float* d_pts32 = nullptr;
    std::vector<Launch> launches;
    std::vector<GenBlock> kblocks;  // K-store layout (near blocks, then far blocks)
    GenBlock* d_kblocks = nullptr;
    int64_t kstore_elems = 0, pstore_elems = 0;
    std::vector<double> pstore_host;  // P and P^T of every node, FP64
    Family fam[2];                    // 0: double, 1: float
    struct TcState* tc = nullptr;     // tensor-core path (eval_tc.cu)
    cudaEvent_t ev[6] = {};
    // CUDA graphs of the launch sequence, keyed by (precision, r, W, ldw, U,
    // ldu): captured on `capture_stream` once a key repeats, replayed on the
    // caller's stream; cleared whenever device buffers are (re)allocated.
    struct GraphEntry {
        int calls = 0;
        int launches = 0;
        cudaGraphExec_t exec = nullptr;
    };
    std::map<std::tuple<int, int64_t, const void*, int64_t, void*, int64_t>, GraphEntry> graphs;
    cudaStream_t capture_stream = nullptr;
    // host-buffer evaluations: copy streams and per-chunk events of the
    // copy / compute pipeline over column chunks of W and U
    cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
    std::vector<cudaEvent_t> pipe_events;
    bool ev_ok = false;
    bool last_fused = false;  // the last tensor-core call ran as one dependency-driven launch
    int last_launches = 0;
};


std::pair<Tile*, int> tiles_for(Launch& l, int bm);

// SIMT evaluation (FP64 / FP32) on caller-supplied scratch (eval.cu).
int simt_evaluate_on(Handle& H, const void* W, int64_t ldw, void* U, int64_t ldu, int r, int precision,
                     cudaStream_t s, void* WT, void* WTIL, void* UTIL);

// tensor-core path (eval_tc.cu)
void tc_prepare(Handle& H, DeviceState& D, int64_t r_max, int precision);
bool tc_ready(const DeviceState& D, int64_t r, int precision);
int tc_run(Handle& H, DeviceState& D, const float* W, int64_t ldw, float* U, int64_t ldu, int r, int precision,
           cudaStream_t s);
void tc_destroy(DeviceState& D);
int tc_error(const DeviceState& D);  // deferred error code of a tensor-core kernel, 0 if none
void tc_clear_error(DeviceState& D);
void tc_stall_next(DeviceState& D, int precision);

}  // namespace gofmm
