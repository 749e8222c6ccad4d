// Internal types of libgofmm: host-side compressed structure, parameters and
// the device-side evaluation plan.  Nothing here is part of the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "gofmm.h"

typedef struct CUstream_st* cudaStream_t;

namespace gofmm {

// Failure carried to the ABI boundary, where it becomes a return code plus
// gofmm_last_error().
struct Error {
    int code;
    std::string msg;
};
[[noreturn]] void fail(int code, const std::string& msg);

// ---------------------------------------------------------------------------
// Counter-based random numbers: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014).
// Output i of the stream keyed by `key` is mix64(key + (i+1) * gamma).  Every
// random choice of the method (centroid samples of Alg. 1, random projection
// splits, ANN recall sample, importance-sampled rows) comes from a stream
// keyed by (seed, purpose, id).
// ---------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
inline uint64_t sm_output(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * kGamma); }
enum Purpose : uint64_t { kCentroid = 1, kAnnSplit = 2, kAnnRecall = 3, kSample = 4, kRandomPerm = 5 };
inline uint64_t stream_key(uint64_t seed, uint64_t purpose, uint64_t sub) {
    return sm_output(seed, (purpose << 40) | sub);
}
// First k entries of a Fisher-Yates shuffle of a driven by the stream `key`
// (step t swaps t with t + (u_t mod (n - t))); `a` is modified in place.
void partial_shuffle(std::vector<int64_t>& a, int64_t k, uint64_t key);

// ---------------------------------------------------------------------------
// Entries of K: generator (Gaussian / IMQ from points) or user callback.
// ---------------------------------------------------------------------------
struct Entries {
    int kind = GOFMM_GEN_CALLBACK;
    int dim = 0;
    int64_t n = 0;
    std::vector<double> pts;  // generator kinds: N x dim
    double h = 1.0, shift = 0.0;
    gofmm_block_fn fn = nullptr;
    void* ctx = nullptr;

    // out[i*nJ + j] = K(I[i], J[j]); throws Error on callback failure or a
    // non-finite entry.
    void block(const int64_t* I, int64_t nI, const int64_t* J, int64_t nJ, double* out) const;
    double diag(int64_t i) const;
    bool is_generator() const { return kind != GOFMM_GEN_CALLBACK; }
};

struct Params {
    int64_t m = 64, s = 64;
    double tau = 1e-5, budget = 0.03;
    int kappa = 32, distance = GOFMM_DIST_GRAM_L2, far_mode = GOFMM_FAR_SYMMETRIC;
    int cache_mode = GOFMM_CACHE_BLOCKS;
    int n_centroid = 32, n_sample = 0, ann_max_iter = 10, num_threads = 0;
    double ann_target_recall = 0.8;
    int64_t knn_exact_max = 16384;
    uint64_t seed = 0;
    int device = 0;
    int sample_device = 0;  // skeletonization blocks K_{I'a} generated on the GPU
};

// ---------------------------------------------------------------------------
// Compressed structure (host, FP64).  Nodes use heap numbering: root 0,
// children 2h+1 and 2h+2, every leaf at depth `depth`.
// ---------------------------------------------------------------------------
struct Structure {
    Params prm;
    int64_t n = 0;
    int depth = 0;
    std::vector<int64_t> perm;            // tree position -> original index
    std::vector<int64_t> node_off;        // per node: first tree position
    std::vector<int64_t> node_size;       // per node: number of indices
    std::vector<std::vector<int64_t>> near;  // per leaf number: leaf numbers (sorted)
    std::vector<std::vector<int64_t>> far;   // per node: far nodes (sorted heap ids)
    std::vector<std::vector<int64_t>> skel;  // per node: skeleton (original indices, pivot order)
    std::vector<std::vector<double>> P;      // per node: s x ncols row-major
    // Blocks cached at compression time for callback matrices (FP64,
    // row-major): near_blocks[b][t] = K(leaf b, Near(b)[t]);
    // far_blocks[h][t] = K(skel h, skel Far(h)[t]).
    std::vector<std::vector<std::vector<double>>> near_blocks, far_blocks;
    int ann_iters = 0;
    double ann_recall = 1.0;
    double compress_seconds = 0.0;

    int64_t n_nodes() const { return (int64_t(2) << depth) - 1; }
    int64_t n_leaves() const { return int64_t(1) << depth; }
    int64_t leaf_node(int64_t b) const { return (int64_t(1) << depth) - 1 + b; }
    bool is_leaf(int64_t h) const { return h >= (int64_t(1) << depth) - 1; }
    int64_t ncols(int64_t h) const {
        return is_leaf(h) ? node_size[h]
                          : int64_t(skel[2 * h + 1].size() + skel[2 * h + 2].size());
    }
};

// Generator entries on the GPU for compression (sample.cu): FP64 blocks
// K(rows, cols), written column-major (m x n, leading dimension m) into host
// memory, for many (rows, cols) pairs per call.
struct SampleJob {
    const int64_t* rows;
    int64_t m;
    const int64_t* cols;
    int64_t n;
    double* out;
};
class DeviceSampler {
public:
    DeviceSampler(const Entries& K, int device);  // uploads the points once
    ~DeviceSampler();
    DeviceSampler(const DeviceSampler&) = delete;
    DeviceSampler& operator=(const DeviceSampler&) = delete;
    // Synchronous: every job's block written to job.out.
    void sample(const std::vector<SampleJob>& jobs);
    // Asynchronous, double-buffered: submit() queues the blocks of a batch
    // (job.out unused) and returns at once; wait(slot) blocks until they are
    // in pinned host memory and returns, per job, a pointer to its block
    // (valid until the slot is submitted again).  At most two batches in
    // flight; submit(b + 1) may run while the caller works on batch b.
    int submit(const std::vector<SampleJob>& jobs);
    std::vector<const double*> wait(int slot);

private:
    struct Slot;
    const Entries& K_;
    int device_;
    double* d_pts_ = nullptr;
    void* stream_ = nullptr;
    Slot* slots_[2] = {nullptr, nullptr};
    int next_ = 0;
};

int tree_depth(int64_t n, int64_t m);
void compress(const Entries& K, Structure& st);  // throws Error
void fill_node_extents(Structure& st);            // node_off/node_size from leaf sizes
void cache_blocks_host(const Entries& K, Structure& st);

// pivoted QR + ID (exposed for tests through the structure only)
struct IdResult {
    std::vector<int64_t> perm;  // pivot order of the columns
    int64_t s = 0;
    std::vector<double> P;      // s x n row-major, original column order
};
IdResult interpolative_decomposition(std::vector<double>& A_colmajor, int64_t m, int64_t n,
                                     int64_t max_rank, double tau);

void export_structure(const Structure& st, const Entries* K, const std::string& path);
void import_structure(const std::string& path, Structure& st);

}  // namespace gofmm

namespace gofmm {

struct DeviceState;  // device-resident plan and workspace (eval.cu)

// Everything a gofmm_handle owns.
struct Handle {
    Structure st;
    Entries K;               // generator kinds keep their points; callbacks are dropped
    DeviceState* dev = nullptr;
    int timing = 0;  // 0 off, 1 one launch per stage with stage events, 2 production path with events
    // tensor-core launch configuration per mode (TF32, BF16, BF16X3), set by
    // the autotuner or by the caller; read when the mode's plan is built
    int tc_piece[3] = {256, 256, 256};  // task piece height (MMA N ceiling): 128 or 256
    int tc_schedule[3] = {0, 0, 0};     // GOFMM_SCHED_FUSED, _STAGED or _PAIR
    int tc_order[3] = {0, 0, 0};        // GOFMM_ORDER_CRITICAL or GOFMM_ORDER_LOCAL (fused schedule)
    int64_t plan_epoch = 0;  // bumped whenever a tensor-core plan is rebuilt (batches check it)
    int64_t inflight = 0;    // engine requests of this handle not yet retired
};

// Device side (eval.cu); all throw Error.
void device_prepare(Handle& H, int64_t r_max, int precision);
// host_buffers: 0 device pointers, 1 host pointers (returns when U is
// written), 2 host pointers, asynchronous (U is final after device_synchronize)
void device_evaluate(Handle& H, const void* W, int64_t ldw, void* U, int64_t ldu, int64_t r,
                     int dtype, int precision, void* stream, int host_buffers);
void device_evaluate_static(Handle& H, const void* W, int64_t ldw, void* U, int64_t ldu, int64_t r, int dtype,
                            int precision, void* stream);
void device_destroy(Handle& H);
void device_synchronize(Handle& H, void* stream);
void device_trim(Handle& H);
void device_stall_next(Handle& H, int precision);

// Tensor-core launch configuration and its autotuner (tune.cu).
constexpr int kTuneMax = 16;  // candidates of one tuning run
struct TuneResult {
    int piece = 256, schedule = 0, order = 0, from_cache = 0, n = 0;
    int cand_piece[kTuneMax] = {}, cand_schedule[kTuneMax] = {}, cand_order[kTuneMax] = {};
    float cand_ms[kTuneMax] = {};
    std::string key;
};
void device_set_tc_config(Handle& H, int precision, int piece, int schedule, int order);
std::string tune_key(const Handle& H, int64_t r, int precision);
std::string tune_key_batch(Handle* const* hs, const int64_t* r, int count, int precision);
TuneResult autotune(Handle& H, int64_t r, int precision, const char* cache_path, void* stream);
TuneResult autotune_batch(Handle* const* hs, const int64_t* r, int count, int precision, const char* cache_path,
                          void* stream);

// Batching / serving engine (engine.cu).
struct Engine;
Engine* engine_create(int device, int precision, int64_t pool_bytes);
int64_t engine_submit(Engine& E, Handle& H, const float* W, int64_t ldw, float* U, int64_t ldu, int64_t r);
int64_t engine_step(Engine& E, cudaStream_t s);
int engine_poll(Engine& E, int64_t id);
int64_t engine_workspace(const Engine& E, Handle& H, int64_t r);
void engine_drain(Engine& E, cudaStream_t s);
void engine_stats(const Engine& E, int64_t* out, int n);
void engine_destroy(Engine* E);

struct Batch;
Batch* batch_create(Handle* const* hs, const int64_t* r, int count, int precision);
int batch_evaluate(Batch& B, const float* const* W, const int64_t* ldw, float* const* U, const int64_t* ldu,
                   cudaStream_t s);
int batch_error(const Batch& B);
void batch_destroy(Batch* B);
void device_stage_times(Handle& H, float* ms, int n);

}  // namespace gofmm
