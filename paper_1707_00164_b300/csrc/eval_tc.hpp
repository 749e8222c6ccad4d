// Tensor-core path: plan, stores and launch interface shared by the
// single-evaluation path (eval_tc.cu) and the batching/serving engine
// (engine.cu).
#pragma once
#include <map>
#include <utility>
#include <vector>

#include "eval_state.hpp"

namespace gofmm {

constexpr int kMaxN = 256;              // MMA N per task (taller tasks are split)
constexpr int kTileBytes = 128 * 128;  // one 128-row x 128-byte operand tile

enum TcMode : int { TC_TF32 = 0, TC_BF16 = 1, TC_BF16X3 = 2 };


struct TcSlab {
    int64_t b_off;     // cached: byte offset of the slab's first chunk tile in the B store;
                       // generated: offset in idx[] of the piece's row list
    int32_t a_buf;     // 0 WT, 1 WTIL, 2 UTIL
    int32_t a_chunk0;  // first chunk of the slab's K range in that RT buffer
    int32_t nchunks;
    int32_t gen;       // 1: the block tiles are generated in the kernel (K(row list, column list))
    int64_t gen_cols;  // generated: offset in idx[] of the column list
    int32_t k;         // generated: columns (the rest of the last chunk is zero)
    int32_t a_node0, a_node1;  // tree nodes whose skeleton rows the slab's right-hand sides are (-1: none)
    // dependency-driven launch: the counters (and arrival counts) the slab's
    // right-hand sides wait for before they are copied (-1: none)
    int32_t dep_c0, dep_n0, dep_c1, dep_n1;
};

struct TcTask {
    int64_t out_pos;  // OUT_U: tree position of row 0; else first chunk of the output segment
    int32_t m;        // valid output rows (<= 256)
    int32_t n_pad;    // MMA N: m rounded up to 16
    int32_t slab0, slab1;
    int32_t out_kind;  // OUT_WTIL, OUT_UTIL, OUT_U
    int32_t accumulate;
    int32_t nchunks;   // chunks over all slabs
    int32_t out_cols;  // RT outputs: columns of the output segment this task writes (zeros past m)
};

struct TcTile {
    int32_t seg, task, rt, pad;  // pad = 2 or 4: r-tiles rt .. rt + pad - 1 (else rt alone)
};

// Tiles of one task over n_rtiles 128-column tiles of r.  Two r-tiles per
// tile feed two accumulators from each staged block stage: fewer staged
// bytes per flop (a third fewer for a 256-row block, a quarter for 128
// rows), and the block is read once per pair of r-tiles.  TMEM holds two
// accumulator buffers of kAccBufCols columns; accumulators of at most
// kAccBufCols / 2 columns share one buffer, so tiles still alternate buffers
// and the epilogue of one overlaps the MMAs of the next: such tasks take two
// r-tiles from kTwoRtMinChunksNarrow chunks on.  Wider accumulators take both
// buffers, which exposes the epilogue: only tasks of kTwoRtMinChunksWide
// chunks or more that write a right-hand-side buffer (the leaves' scattered
// U rows are slower to write) take two r-tiles then.
constexpr int kAccBufCols = 256;
constexpr int kTwoRtMinChunksNarrow = 4;
constexpr int kTwoRtMinChunksWide = 16;
// wmax = 4 (the generator variant of the 128-row kernel, whose stages hold
// four r-tiles): narrow tasks take four r-tiles per tile where four remain,
// filling both accumulator buffers; the block stage (generated in the
// kernel) then serves four r-tiles.
inline void task_tiles(std::vector<TcTile>& out, int32_t seg, int32_t task, const TcTask& tk, int n_rtiles,
                       int wmax = 2) {
    const bool narrow = 2 * tk.n_pad <= kAccBufCols;
    const bool two = narrow ? tk.nchunks >= kTwoRtMinChunksNarrow
                            : tk.nchunks >= kTwoRtMinChunksWide && tk.out_kind != OUT_U;
    const bool four = wmax >= 4 && narrow && two;
    for (int rt = 0; rt < n_rtiles;) {
        const int w = four && rt + 3 < n_rtiles ? 4 : two && rt + 1 < n_rtiles ? 2 : 1;
        out.push_back(TcTile{seg, task, int32_t(rt), int32_t(w)});
        rt += w;
    }
}
// r-tiles of a tile (TcTile::pad)
inline int tile_width_host(const TcTile& t) { return t.pad == 2 || t.pad == 4 ? t.pad : 1; }

// One (evaluation, launch) pair inside a tensor-core launch: the tasks and
// slabs of that launch of one compressed matrix, its B tiles, the RT buffers
// of that evaluation, and its output.
struct TcSeg {
    const TcTask* tasks;
    const TcSlab* slabs;
    const uint8_t* b_hi;
    const uint8_t* b_lo;
    uint8_t* rt_hi[3];
    uint8_t* rt_lo[3];
    int64_t rt_chunks[3];
    float* U;
    int64_t ldu;
    const int64_t* perm;
    int32_t r;
    int32_t tile_base;    // segment tile lists: first global tile index of this segment
    const TcTile* tiles;  // segment tile lists (TcParams::tiles == nullptr): this segment's tiles
    // in-kernel entry generation (generated slabs): point table in index-list
    // order (row t = the point of perm[t], tree order then skeleton lists),
    // dpad floats per point (the coordinates, then the point's squared norm,
    // then zeros to a multiple of 4);
    // GOFMM_GEN_GAUSSIAN exp(-d2 inv) or GOFMM_GEN_IMQ 1/sqrt(1 + d2 inv),
    // plus shift where the row and column are the same index-list position
    const float* pts;
    int32_t dim, dpad, gen_kind, pad2;
    float gen_inv, gen_shift;
    // dependency-driven launch (TcParams::tile_next set and dep_off not
    // null; a launch without dependencies leaves all five null): tile
    // (task, rt) waits until counters[c * dep_nrt + rt] >= e for every (c, e) in
    // deps[dep_off[task] .. dep_off[task+1]) and for its slabs' operand
    // counters, and adds one to counters[sig[2 task + i] * dep_nrt + rt]
    // (i = 0, 1; -1 = none) per epilogue warp when done
    const int32_t* dep_off;
    const int32_t* deps;
    const int32_t* sig;
    int* counters;
    int32_t dep_nrt, pad3;
};
constexpr int kGenMaxDpad = 16;  // generated blocks: at most 16 floats per point (15 coordinates and the norm)
constexpr int kMaxSegs = 64;  // segments per launch (kernel parameters, by value)
constexpr int kClaimSlots = 64;  // per-stage launches of one evaluation that claim tiles dynamically


// Ready queue of a dependency-driven launch of one evaluation (order
// GOFMM_ORDER_READY).  The tiles tiles[0 .. n_static) are claimed in list
// order; the tiles tiles[n_static .. n_static + n) (the downward pushes,
// where a plan has them, and the leaves) only through a FIFO that holds a
// tile once every counter it
// waits for is complete: the epilogue that brings a counter to its final
// arrival count req[c] takes one from the pending count of each queued tile
// waiting on it (cons) and appends the tiles that reach zero.  A producer
// takes a ready tile first, else the next tile of the list, else (list
// exhausted) waits for the next queue slot.  All ints, reset before every
// launch: queue = {tail (slots reserved), head (slots claimed), n entries,
// -1 until written}, pending = the initial counts.
struct TcReady {
    int* queue;
    int* pending;
    const int32_t* cons_off;  // [ncounters * r-tiles + 1]
    const int32_t* cons;      // queued-tile numbers (0 .. n) waiting on (counter, r-tile)
    const int32_t* req;       // [ncounters]: arrivals that complete a counter
    int n_static, n;
};

struct TcParams {
    const TcTile* tiles;  // merged tile list; nullptr: every segment brings its own (TcSeg::tiles)
    int ntiles;
    int nsegs;
    int* err;
    // tiles are taken in list order from this zeroed counter by whichever
    // CTA is free (dynamic; with dependency waits in the segments that carry
    // dependency arrays, which needs every CTA resident: a cooperative
    // launch); nullptr: static round-robin split, no waits
    int* tile_next;
    TcReady ready;  // queue == nullptr: no ready queue
    TcSeg segs[kMaxSegs];
};

// Conversion of one row-major FP32 block (plan store) into its B tiles.
// col_map_off >= 0: destination column c of the tile takes source column
// col_maps[col_map_off + c] (-1: zero) instead of the k_split / k_gap rule.
struct TileJob {
    int64_t src_off, dst_off, col_map_off;
    int32_t src_ld, m, k, n_pad, nchunks, k_split, k_gap, src_store;
};

struct TcLaunch {
    std::vector<TcTask> tasks;
    std::vector<TcSlab> slabs;
    std::vector<int64_t> task_node;  // node each task writes (host only)
    TcTask* d_tasks = nullptr;
    TcSlab* d_slabs = nullptr;
    int stage = 0;
    int piece = 256;  // task piece height of the plan
    int wmax = 2;     // r-tiles per tile at most in a launch of this plan's own kernel (task_tiles)
    std::map<int, std::pair<TcTile*, int>> tiles;  // r-tiles, order, form -> tile list of this launch alone
};

// Every grouped GEMM of one evaluation as one dependency-driven launch.
struct TcFused {
    std::vector<TcTask> tasks;
    std::vector<TcSlab> slabs;
    std::vector<int32_t> order;        // tasks in a topological, critical-path-first order
    std::vector<int32_t> order_local;  // topological; groups by critical path, heap order inside
    std::vector<int32_t> order_sched;  // a simulated list schedule's order (topological)
    std::vector<int32_t> order_levels;  // S2S top-down (push levels, if any, one S2S level later), then leaves
    int piece = 256;                   // task piece height of the plan
    int wmax = 2;                      // r-tiles per tile at most (task_tiles)
    TcTask* d_tasks = nullptr;
    TcSlab* d_slabs = nullptr;
    int32_t* d_dep_off = nullptr;
    int32_t* d_deps = nullptr;
    int32_t* d_sig = nullptr;
    int ncounters = 0;
    int* d_counters = nullptr;  // ncounters x r-tiles of the largest r prepared (+ tile counter)
    int counters_nrt = 0;
    std::vector<int32_t> deps_host;
    // host copies for the ready-queue tile lists: task-level dependency
    // offsets, each task's stage, and the (counter, count) pairs of its slabs
    std::vector<int32_t> dep_off_host;
    std::vector<int8_t> task_stage;
    // ready-queue form per r-tile count: tiles (list part, then queued part)
    // and the device arrays of TcReady (queue and pending reset per launch
    // from their initial copies)
    struct Ready {
        TcTile* tiles = nullptr;
        int n_static = 0, n = 0;
        int* queue = nullptr;
        int* queue0 = nullptr;
        int* pending = nullptr;
        int* pending0 = nullptr;
        int32_t* cons_off = nullptr;
        int32_t* cons = nullptr;
        int32_t* req = nullptr;
    };
    std::map<int, Ready> ready;
    int32_t* d_deps_stall = nullptr;  // diagnostic copies with one unreachable arrival count
    TcSlab* d_slabs_stall = nullptr;
    bool stall_next = false;
    std::map<int, std::pair<TcTile*, int>> tiles;  // 2 x r-tiles + order -> ordered tile list
};

struct TcPrec {
    int mode = 0, kc = 0, es = 0;
    int piece = kMaxN;  // task piece height: tasks taller than this are split (MMA N ceiling)
    bool gen = false;   // some slabs generate their block tiles in the kernel (no cached blocks)
    float* gen_pts = nullptr;  // generator: point table (index-list order), kind, 1/(2h^2) or 1/h^2, shift
    int gen_dim = 0, gen_dpad = 0, gen_kind = 0;
    float gen_inv = 0.f, gen_shift = 0.f;
    bool split = false;
    std::vector<TcLaunch> launches;
    int64_t wt_chunks = 0, sk_chunks = 0;
    int64_t* d_chunk_pos = nullptr;    // WT chunk -> tree position of its first row
    int32_t* d_chunk_valid = nullptr;  // WT chunk -> valid rows
    uint8_t* b_hi = nullptr;
    uint8_t* b_lo = nullptr;
    int64_t b_bytes = 0;
    int64_t r_cap = 0;  // right-hand sides the RT buffers hold (multiple of 128)
    uint8_t* rt_hi[3] = {nullptr, nullptr, nullptr};
    uint8_t* rt_lo[3] = {nullptr, nullptr, nullptr};
    int* d_err = nullptr;
    int* h_err = nullptr;  // pinned
    int num_sms = 148;     // persistent grid size
    int* d_claims = nullptr;  // tile counters of the per-stage launches of one evaluation (kClaimSlots)
    TcFused fused;       // every stage in one launch
    TcFused fused_up;    // N2S levels in one launch (hybrid schedule)
    TcFused fused_down;  // S2N levels and leaves in one launch (hybrid schedule)
};

struct TcState {
    TcPrec* prec[3] = {nullptr, nullptr, nullptr};
};


int mode_of(int precision);
TcPrec& tc_plan(Handle& H, DeviceState& D, int precision);  // plan + B tiles (allocates, synchronises)
TcSeg make_seg(const TcPrec& T, const TcLaunch& l, uint8_t* const* rt_hi, uint8_t* const* rt_lo, float* U,
               int64_t ldu, const int64_t* perm, int r);
void launch_gemm_mode(int mode, int piece, const TcParams& p, int num_sms, cudaStream_t s, bool gen = false);
// cooperative launch (every CTA resident): the dependency-driven mode
void launch_gemm_coop_mode(int mode, int piece, const TcParams& p, int num_sms, cudaStream_t s, bool gen);
// the fused plan's task order for a GOFMM_ORDER_* value
inline const std::vector<int32_t>& fused_order(const TcFused& F, int order) {
    // (the ready-queue form takes its list part from the locality order; a
    // batch, which has no ready queue, runs it as the locality order)
    return order == GOFMM_ORDER_LOCAL || order == GOFMM_ORDER_READY ? F.order_local
           : order == GOFMM_ORDER_SCHEDULE                        ? F.order_sched
           : order == GOFMM_ORDER_LEVELS                          ? F.order_levels
                                                                  : F.order;
}
// device tile list of one launch alone for n_rtiles r-tiles (cached in the launch)
std::pair<TcTile*, int> launch_tiles(TcLaunch& l, int n_rtiles, int order, bool pair = false, int wmax = 2);
void tc_drop_plan(DeviceState& D, int precision);  // frees one mode's plan, stores and buffers
void launch_gather(int mode, const TcPrec& T, const float* W, int64_t ldw, const int64_t* perm, uint8_t* wt_hi,
                   uint8_t* wt_lo, int r, cudaStream_t s);

}  // namespace gofmm
