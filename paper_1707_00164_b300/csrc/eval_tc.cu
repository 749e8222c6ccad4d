// Tensor-core evaluation path for sm_103a: tcgen05.mma (TF32, BF16, split
// BF16x3 with FP32 accumulation) on operands staged in shared memory by bulk
// copies, accumulators in tensor memory (TMEM).
//
// Formulation.  Every grouped-GEMM task of the evaluation plan computes
//     out[m x r] = sum_slabs A_slab[m x k] * B_slab[k x r]
// (A: a cached K block, an interpolation matrix P or P^T; B: rows of a
// right-hand-side buffer).  On the tensor cores it runs transposed,
//     out^T[r x m] = sum_slabs B_slab^T[r x k] * A_slab^T[k x m],
// so the 128-row MMA dimension M is a tile of the r right-hand sides (always
// full) and the ragged block height m (a skeleton or leaf size) is the MMA's
// N (padded to a multiple of 16, at most 256; taller tasks are split).
// Both MMA operands are K-major:
//   MMA A = right-hand sides in "RT" layout: for every 128 columns of r and
//           every chunk of KC rows (128 bytes of K), one 128 x 128 B tile;
//           node segments are padded to whole chunks (padding stays zero);
//   MMA B = the blocks, per block and chunk one n_pad x 128 B tile.
// A chunk tile is stored as its two K-halves (rows x 64 B each, 64-byte
// swizzle), one after the other.  Every half sits in HBM exactly as the MMA
// reads it from shared memory, so a single linear cp.async.bulk stages it
// (no tensor maps).
//
// Kernel: persistent, one CTA per SM looping over tiles (a task and one or
// two 128-column tiles of r), 6 warps.  Warp 0 streams stages into a ring
// in shared memory (mbarrier complete_tx): one K-half of a chunk (split
// BF16x3) or a whole chunk (TF32, BF16) of the block and of the tile's one
// or two right-hand-side tiles, 64 KB.  Warp 1 allocates TMEM (two
// 256-column accumulator buffers) and one thread issues the MMAs, the block
// against each right-hand-side tile into its own accumulator (a two-r-tile
// tile stages the block once for both), and commits each stage back to the
// producer.  Warps 2-5 read finished accumulators (tcgen05.ld) while the
// MMAs of the next tile run and write the outputs: the next stage's RT
// operand (rounded to TF32 / BF16 / BF16 hi+lo; a fresh segment through a
// shared-memory staging tile and bulk stores) or, for the leaves, U
// scattered to the original order in FP32.  Every wait is bounded; on
// timeout the kernel records an error code, drains what it issued and
// returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <queue>
#include <set>
#include <tuple>

#include "eval_tc.hpp"

namespace gofmm {

int mode_of(int precision) {
    return precision == GOFMM_PREC_TF32 ? TC_TF32 : precision == GOFMM_PREC_BF16 ? TC_BF16 : TC_BF16X3;
}

namespace {

constexpr long long kSpinLimit = 2000000000LL;  // clock cycles (about a second) before a wait gives up
constexpr int kErrProducer = 1, kErrMma = 2, kErrEpilogue = 3, kErrDependency = 4, kErrTmemPair = 5,
              kErrGenerator = 6;
constexpr int kGenWarps = 8;      // generator warps of the in-kernel entry generation
constexpr int kGenThreads = 192 + 32 * kGenWarps;  // threads of the kernel variant with generator warps

// One stage of a generated block tile: rows perm[rows .. rows + m) (the
// rest of the n_pad rows zero), columns perm[cols .. cols + kvalid) (the rest
// of the stage zero), written into stage `stage`.  The columns' points reach
// the job's slot of the column-point ring by a bulk copy that completes on
// the job's barrier.
struct GenJob {
    int64_t rows, cols;
    int32_t seg, stage, m, kvalid, n_pad, stop;
};

// NMAX: the tallest task piece the kernel accepts (MMA N ceiling, 128 or
// 256).  A stage holds one K-half of a chunk (64 bytes of every row): the
// halves of two 128-row right-hand-side tiles and of one NMAX-row block tile
// (twice for split BF16x3); as many stages as fit in about 200 KB of shared
// memory, so a lower ceiling buys a deeper pipeline.
template <int MODE, int NMAX = kMaxN, int W = 2>
struct Cfg {
    static constexpr bool kSplit = MODE == TC_BF16X3;
    // K-halves per stage: one for split BF16x3 (a stage of two r-tiles and a
    // 256-row block is then 64 KB), both (the whole chunk) otherwise
    static constexpr int kSub = kSplit ? 1 : 2;
    static constexpr int kHalfA = 128 * 64;      // one K-half of a right-hand-side tile
    static constexpr int kAUnit = kSub * kHalfA;  // one r-tile's part of a stage
    static constexpr int kW = W;                  // r-tiles a stage can hold
    static constexpr int kPart = kW * kAUnit + kSub * NMAX * 64;  // hi (or lo) part of a stage
    static constexpr int kStageBytes = (kSplit ? 2 : 1) * kPart;
    static constexpr int kStages = (200 * 1024 / kStageBytes) < 8 ? (200 * 1024 / kStageBytes) : 8;
    static constexpr int kSmem = kStages * kStageBytes + 1024 + 256;  // + alignment slack, barriers
    static constexpr int kKc = MODE == TC_TF32 ? 32 : 64;  // columns per chunk
    static constexpr int kStageK = kKc / 2 * kSub;          // columns per stage
    static constexpr int kEs = MODE == TC_TF32 ? 4 : 2;
    static constexpr int kTmemCols = 2 * kAccBufCols;  // two accumulator buffers
    static_assert(kStages >= 2, "at least a double-buffered stage ring");
    // epilogue staging tile (hi and lo) of the kernels without generator warps
    static constexpr int kEpiBytes = (kSplit ? 2 : 1) * kTileBytes;
    static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
    // generator warps' area: barriers, flags and the job ring (1 KB), then
    // one slot of column points per job (kStageK points of up to 16 floats)
    static constexpr int kColSlot = kStageK * kGenMaxDpad * 4;
    static constexpr int kGenBytes = 1024 + kStages * kColSlot;
    static_assert(kSmem + kGenBytes <= 227 * 1024, "shared memory per CTA with generator warps");
    static_assert(kSmem + kEpiBytes <= 227 * 1024, "shared memory per CTA with the epilogue staging tile");
};
// Stage layout of tc_gemm_kernel<MODE, NMAX, GEN>: the generator variant of
// the 128-row kernel holds four r-tiles per stage, so a tile can cover four
// r-tiles and each generated block stage serves all of them (each block is
// generated once per four r-tiles instead of once per two).
template <int MODE, int NMAX, bool GEN>
using KCfg = Cfg<MODE, NMAX, (GEN && NMAX == 128) ? 4 : 2>;
// dynamic shared memory of tc_gemm_kernel<MODE, NMAX, GEN>
template <int MODE, int NMAX, bool GEN>
constexpr int gemm_smem() {
    return KCfg<MODE, NMAX, GEN>::kSmem + (GEN ? KCfg<MODE, NMAX, GEN>::kGenBytes : KCfg<MODE, NMAX, GEN>::kEpiBytes);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Polls between two looks at the grid's error flag in a bounded wait: the
// flag is a global load (an L2 round trip), so reading it after every poll
// would delay noticing the phase change by that round trip.
constexpr uint32_t kPollsPerCheck = 64;
// Bounded wait on an mbarrier phase; false (and an error code recorded) on
// timeout or when another thread of the grid already failed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it % kPollsPerCheck == 0) {
            if (*reinterpret_cast<volatile int*>(err) != 0) return false;
            if (clock64() - t0 > kSpinLimit) {
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}
// Bounded wait until *ctr >= e (acquire); false on timeout or a recorded error.
__device__ __forceinline__ bool wait_counter(const int* ctr, int e, int* err) {
    const long long t0 = clock64();
    for (uint32_t it = 1;; ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= e) return true;
        if (it % 16 == 0) {
            if (*reinterpret_cast<volatile int*>(err) != 0) return false;
            if (clock64() - t0 > kSpinLimit) {
                atomicCAS(err, 0, kErrDependency);
                return false;
            }
        }
        __nanosleep(64);
    }
}
__device__ __forceinline__ int ld_acquire_i32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_i32(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Ready queue (TcReady): the tile written into a claimed slot, after a
// bounded wait for its writer; -1 on timeout or a recorded error.
__device__ __noinline__ int ready_entry(const TcParams& p, int slot) {
    const int* e = p.ready.queue + 2 + slot;
    const long long t0 = clock64();
    for (uint32_t it = 1;; ++it) {
        const int v = ld_acquire_i32(e);
        if (v >= 0) return v;
        if (it % 16 == 0) {
            if (*reinterpret_cast<volatile int*>(p.err) != 0) return -1;
            if (clock64() - t0 > kSpinLimit) {
                atomicCAS(p.err, 0, kErrDependency);
                return -1;
            }
        }
        __nanosleep(64);
    }
}
// Next tile of a ready-queue launch: a queued tile whose inputs are
// complete, else the next tile of the list, else (the list exhausted) the
// next queue slot, waited for.  -1: no tile left, or an error.  No CTA takes
// a queued slot it has to wait for while the list still has tiles, and
// every queued tile is written into exactly one slot, so a waiting CTA is
// always served.
__device__ __noinline__ int ready_claim(const TcParams& p, bool& list_left) {
    int* q = p.ready.queue;  // q[0]: slots reserved by writers, q[1]: slots claimed
    for (;;) {
        const int head = *reinterpret_cast<volatile int*>(q + 1);
        const int tail = ld_acquire_i32(q);
        if (head < tail) {
            if (atomicCAS(q + 1, head, head + 1) == head) return ready_entry(p, head);
            continue;
        }
        if (list_left) {
            const int s = atomicAdd(p.tile_next, 1);
            if (s < p.ready.n_static) return s;
            list_left = false;
            continue;
        }
        const int h = atomicAdd(q + 1, 1);
        return h < p.ready.n ? ready_entry(p, h) : -1;
    }
}
// The arrival that completed counter pair `pair` (counter * r-tiles + r-tile):
// every queued tile waiting on it loses one pending count; those that reach
// zero are appended to the queue.
__device__ __noinline__ void ready_release(const TcParams& p, int pair) {
    __threadfence();  // the earlier arrivals on this counter happen before the entries written below
    for (int i = p.ready.cons_off[pair]; i < p.ready.cons_off[pair + 1]; ++i) {
        const int u = p.ready.cons[i];
        if (atomicSub(p.ready.pending + u, 1) == 1) {
            const int slot = atomicAdd(p.ready.queue, 1);
            st_release_i32(p.ready.queue + 2 + slot, p.ready.n_static + u);
        }
    }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups
// 512 bytes apart (tile rows at a 64-byte stride).
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFFu) >> 4);  // start address
    d |= uint64_t(1) << 16;                   // leading byte offset (unused when swizzled)
    d |= uint64_t(512 >> 4) << 32;            // stride byte offset
    d |= uint64_t(1) << 46;                   // descriptor version
    d |= uint64_t(4) << 61;                   // 64-byte swizzle
    return d;
}
// Instruction descriptor (kind::tf32 / kind::f16): FP32 accumulator, both
// operands K-major, M = 128.
__device__ __forceinline__ uint32_t make_idesc(int fmt, int n) {
    return (1u << 4) | (uint32_t(fmt) << 7) | (uint32_t(fmt) << 10) | (uint32_t(n >> 3) << 17) |
           (uint32_t(128 >> 4) << 24);
}
template <int MODE>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    if constexpr (MODE == TC_TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
    }
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ float round_tf32(float x) {
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return __uint_as_float(y);
}
// Operand tile layout.  A chunk tile (rows x 128 bytes: kc columns of every
// row) is stored as two K-halves, each rows x 64 bytes with the 64-byte
// swizzle (16-byte group g of row n at group g ^ ((n >> 1) & 3)), so one
// half is one contiguous copy and one shared-memory stage.
// byte position of (row, byte-in-row < 64) inside one half
__device__ __forceinline__ uint32_t swz64(uint32_t row, uint32_t byte) {
    return row * 64u + ((((byte >> 4) ^ ((row >> 1) & 3u)) << 4) | (byte & 15u));
}
// byte position of (row, byte-in-row < 128) inside a chunk tile of `rows` rows
__device__ __forceinline__ uint32_t swz(uint32_t row, uint32_t byte, uint32_t rows) {
    return (byte >> 6) * rows * 64u + swz64(row, byte & 63u);
}
// Rows of r-tile rt of a right-hand-side (RT) tile that carry columns of r:
// r rounded up to 16, minus the r-tiles before, at most 128.  Only these
// rows are written (zeros from r on) and copied into shared memory, so a
// K-half moves rt_rows * 64 bytes, a prefix of whole 8-row swizzle groups.
// The stale rows past them in a stage only reach accumulator lanes of
// columns j >= r (a lane of a transposed product is one column of r), and
// nothing writes those lanes out.
__device__ __forceinline__ int rt_rows(int r, int rt) {
    const int v = ((r + 15) & ~15) - rt * 128;
    return v < 0 ? 0 : v > 128 ? 128 : v;
}


__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Named barrier 2 over the four epilogue warps, and its reduction form
// (true iff every epilogue thread passes true).
__device__ __forceinline__ void epi_bar_sync() { asm volatile("bar.sync 2, 128;" ::: "memory"); }
__device__ __forceinline__ int epi_bar_and(bool pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 2, 128, p;\n\tselp.b32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(int(pred))
        : "memory");
    return r;
}
// Bulk store shared -> global (16-byte aligned, size a multiple of 16) and
// its completion waits: .read = the source may be overwritten; plain = the
// writes are performed.
__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Tile t of a launch: from the merged list, or (segment tile lists) from the
// list of the segment whose range holds t.
__device__ __forceinline__ TcTile fetch_tile(const TcParams& p, int t) {
    if (p.tiles) return p.tiles[t];
    int k = 0;
    while (k + 1 < p.nsegs && t >= p.segs[k + 1].tile_base) ++k;
    TcTile tt = p.segs[k].tiles[t - p.segs[k].tile_base];
    tt.seg = k;
    return tt;
}
// r-tiles a tile covers: rt alone, or rt .. rt + 1 (rt .. rt + 3) with two
// (four) accumulators fed from one block stage
__device__ __forceinline__ int tile_width(const TcTile& tt) { return tt.pad == 2 || tt.pad == 4 ? tt.pad : 1; }
// TMEM accumulator buffers (kAccBufCols columns each) a tile takes: one, or
// both when it has two accumulators of more than kAccBufCols / 2 columns or
// four (narrower ones share a buffer, at columns 0 and kAccBufCols / 2)
__device__ __forceinline__ int acc_buffers(int nw, int n_pad) {
    return nw == 4 || (nw == 2 && 2 * n_pad > kAccBufCols) ? 2 : 1;
}
// TMEM columns between the accumulators of consecutive r-tiles of a tile:
// a buffer each, or half a buffer (two per buffer; four r-tiles of at most
// kAccBufCols / 2 columns fill both buffers)
__device__ __forceinline__ int acc_stride(int nw, int nb) { return nb == 2 && nw == 2 ? kAccBufCols : kAccBufCols / 2; }
// Row form of a tile (split BF16x3 only): a two-r-tile tile of a leaf task
// (U rows, at most 128 of them) runs as ONE M = 128, N = 256 product per K
// step, block rows x the two r-tiles' right-hand sides (the block as the A
// operand, the two adjacent r-tile halves of the stage as one 256-row B
// operand), instead of two M = 128 (r-tile) x N = n_pad products that each
// read the block again: a quarter fewer shared-memory operand bytes per
// flop.  The accumulator is then block row x r (TMEM lane = U row).
__device__ __forceinline__ bool row_form(const TcTask& tk, int nw, bool split) {
    return split && nw == 2 && tk.out_kind == OUT_U && !tk.accumulate && tk.n_pad <= 128;
}

// Epilogue of one tile: the accumulator rows of this thread (one column j
// of r) for the task's n_pad block rows, read from TMEM at taddr and written
// as U rows (scattered to the original order, FP32) or as the next stage's
// RT operand (rounded to the mode's format, hi/lo for split BF16).
template <int MODE>
__device__ __forceinline__ void write_tile(const TcSeg& sg, const TcTask& tk, int rt, int row, uint32_t taddr) {
    using C = Cfg<MODE>;
    const int j = rt * 128 + row;
    const bool jv = j < sg.r;
    const int lane = row & 31;
    const int ncols = tk.out_kind == OUT_U ? tk.n_pad : (tk.accumulate ? tk.n_pad : tk.out_cols);
    for (int n0 = 0; n0 < ncols; n0 += 32) {
        float v[32];
        if (tk.nchunks > 0 && n0 < tk.n_pad) {
            tmem_ld32(taddr + uint32_t(n0), v);
#pragma unroll
            for (int e = 0; e < 32; ++e)
                if (n0 + e >= tk.n_pad || !jv) v[e] = 0.f;  // TMEM past n_pad is not this tile's
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = 0.f;
        }
        if (tk.out_kind == OUT_U) {
            // U rows perm[out_pos + n0 .. + 32): lane l loads the row index of
            // n0 + l, the warp shares them by shuffles; all loads of the 32
            // rows are issued before the first add (one latency, not 32)
            const int nl = n0 + lane;
            const int64_t prow = nl < tk.m ? sg.perm[tk.out_pos + nl] : 0;
#pragma unroll
            for (int e0 = 0; e0 < 32; e0 += 16) {  // 16 rows at a time (registers)
                float old[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int64_t pr = __shfl_sync(0xffffffffu, prow, e0 + e);
                    old[e] = (tk.accumulate && jv && n0 + e0 + e < tk.m) ? sg.U[pr * sg.ldu + j] : 0.f;
                }
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int64_t pr = __shfl_sync(0xffffffffu, prow, e0 + e);
                    if (jv && n0 + e0 + e < tk.m)
                        sg.U[pr * sg.ldu + j] = tk.accumulate ? old[e] + v[e0 + e] : v[e0 + e];
                }
            }
            continue;
        }
        // RT rows past rt_rows are never read: an accumulating output skips
        // the rows j >= r, a fresh output writes zeros up to r rounded to 16
        if (tk.accumulate ? !jv : row >= rt_rows(sg.r, rt)) continue;
        // RT output: 32 consecutive k of this row, inside one chunk
        const int buf = tk.out_kind == OUT_WTIL ? 1 : 2;
        const int64_t chunk = tk.out_pos + n0 / C::kKc;
        const uint32_t byte0 = uint32_t((n0 % C::kKc) * C::kEs);
        uint8_t* thi = sg.rt_hi[buf] + (int64_t(rt) * sg.rt_chunks[buf] + chunk) * kTileBytes;
        if constexpr (MODE == TC_TF32) {
            // accumulating: every existing 16-byte group loaded first
            float4 ex[8];
#pragma unroll
            for (int piece = 0; piece < 8; ++piece) {
                ex[piece] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (tk.accumulate && n0 + 4 * piece < tk.n_pad)
                    ex[piece] = *reinterpret_cast<const float4*>(thi + swz(row, byte0 + piece * 16, 128));
            }
#pragma unroll
            for (int piece = 0; piece < 8; ++piece) {
                if (tk.accumulate && n0 + 4 * piece >= tk.n_pad) break;
                float4* dst = reinterpret_cast<float4*>(thi + swz(row, byte0 + piece * 16, 128));
                float4 o = make_float4(v[4 * piece], v[4 * piece + 1], v[4 * piece + 2], v[4 * piece + 3]);
                if (tk.accumulate) {
                    o.x += ex[piece].x; o.y += ex[piece].y; o.z += ex[piece].z; o.w += ex[piece].w;
                }
                *dst = make_float4(round_tf32(o.x), round_tf32(o.y), round_tf32(o.z), round_tf32(o.w));
            }
        } else {
            uint8_t* tlo = C::kSplit ? sg.rt_lo[buf] + (int64_t(rt) * sg.rt_chunks[buf] + chunk) * kTileBytes
                                     : nullptr;
            // accumulating: every existing 16-byte group (hi and lo) loaded first
            uint4 eh[4], el[4];
#pragma unroll
            for (int piece = 0; piece < 4; ++piece) {
                eh[piece] = make_uint4(0, 0, 0, 0);
                el[piece] = make_uint4(0, 0, 0, 0);
                if (tk.accumulate && n0 + 8 * piece < tk.n_pad) {
                    const uint32_t pos = swz(row, byte0 + piece * 16, 128);
                    eh[piece] = *reinterpret_cast<const uint4*>(thi + pos);
                    if constexpr (C::kSplit) el[piece] = *reinterpret_cast<const uint4*>(tlo + pos);
                }
            }
#pragma unroll
            for (int piece = 0; piece < 4; ++piece) {
                if (tk.accumulate && n0 + 8 * piece >= tk.n_pad) break;
                const uint32_t pos = swz(row, byte0 + piece * 16, 128);
                const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&eh[piece]);
                const __nv_bfloat16* l = reinterpret_cast<const __nv_bfloat16*>(&el[piece]);
                uint4 oh, ol;
                __nv_bfloat16* hh = reinterpret_cast<__nv_bfloat16*>(&oh);
                __nv_bfloat16* ll = reinterpret_cast<__nv_bfloat16*>(&ol);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    float x = v[8 * piece + e];
                    if (tk.accumulate) x += __bfloat162float(h[e]) + (C::kSplit ? __bfloat162float(l[e]) : 0.f);
                    hh[e] = __float2bfloat16_rn(x);
                    ll[e] = __float2bfloat16_rn(x - __bfloat162float(hh[e]));
                }
                *reinterpret_cast<uint4*>(thi + pos) = oh;
                if constexpr (C::kSplit) *reinterpret_cast<uint4*>(tlo + pos) = ol;
            }
        }
    }
}

// Epilogue of a row-form tile: this thread's accumulator lane is block row
// n of the task, its 256 columns the r-tiles rt and rt + 1; written as U row
// perm[out_pos + n] (FP32), 16 bytes per store where U allows it.
__device__ __forceinline__ void write_rows(const TcSeg& sg, const TcTask& tk, int rt, int n, uint32_t taddr) {
    const bool rv = n < tk.m;
    float* urow = sg.U + (rv ? sg.perm[tk.out_pos + n] : 0) * sg.ldu;
    const bool vec = ((reinterpret_cast<uintptr_t>(sg.U) | (uintptr_t(sg.ldu) * 4u)) & 15u) == 0;
    for (int c0 = 0; c0 < 2 * 128; c0 += 32) {
        const int j0 = rt * 128 + c0;
        if (j0 >= sg.r) break;  // the same for the whole warp
        float v[32];
        tmem_ld32(taddr + uint32_t(c0), v);
        if (!rv) continue;
        if (vec && j0 + 32 <= sg.r) {
#pragma unroll
            for (int e = 0; e < 32; e += 4)
                *reinterpret_cast<float4*>(urow + j0 + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e)
                if (j0 + e < sg.r) urow[j0 + e] = v[e];
        }
    }
}

// Epilogue of one tile whose output is a fresh RT segment (no accumulation):
// chunk by chunk, the four epilogue warps write their rows into the staging
// tile in the operand layout (zeros in the padding columns and in rows
// r .. rt_rows) and one thread stores the tile's rt_rows leading rows of
// each K-half (the whole 16 KB chunk tile when they are all 128), and its lo
// copy, with bulk copies.  The store thread waits for the previous chunk's
// copies to have read the staging tile before it is written again.
template <int MODE>
__device__ __forceinline__ void write_tile_staged(const TcSeg& sg, const TcTask& tk, int rt, int row, uint32_t taddr,
                                                  uint8_t* stg, bool store_thread) {
    using C = Cfg<MODE>;
    const int j = rt * 128 + row;
    const bool jv = j < sg.r;
    const int buf = tk.out_kind == OUT_WTIL ? 1 : 2;
    const int rows = rt_rows(sg.r, rt);  // rows of the tile that are stored
    const bool rw = row < rows;
    for (int ch = 0; ch * C::kKc < tk.out_cols; ++ch) {
        if (store_thread) bulk_wait_read();
        epi_bar_sync();
#pragma unroll
        for (int h = 0; h < C::kKc; h += 32) {  // 32 columns per TMEM load
            const int n0 = ch * C::kKc + h;
            float v[32];
            if (tk.nchunks > 0 && n0 < tk.n_pad) {
                tmem_ld32(taddr + uint32_t(n0), v);
#pragma unroll
                for (int e = 0; e < 32; ++e)
                    if (n0 + e >= tk.n_pad || !jv) v[e] = 0.f;
            } else {
#pragma unroll
                for (int e = 0; e < 32; ++e) v[e] = 0.f;
            }
            const uint32_t byte0 = uint32_t(h * C::kEs);
            if (!rw) continue;
            if constexpr (MODE == TC_TF32) {
#pragma unroll
                for (int piece = 0; piece < 8; ++piece)
                    *reinterpret_cast<float4*>(stg + swz(row, byte0 + piece * 16, 128)) =
                        make_float4(round_tf32(v[4 * piece]), round_tf32(v[4 * piece + 1]),
                                    round_tf32(v[4 * piece + 2]), round_tf32(v[4 * piece + 3]));
            } else {
#pragma unroll
                for (int piece = 0; piece < 4; ++piece) {
                    uint4 oh, ol;
                    __nv_bfloat16* hh = reinterpret_cast<__nv_bfloat16*>(&oh);
                    __nv_bfloat16* ll = reinterpret_cast<__nv_bfloat16*>(&ol);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        hh[e] = __float2bfloat16_rn(v[8 * piece + e]);
                        ll[e] = __float2bfloat16_rn(v[8 * piece + e] - __bfloat162float(hh[e]));
                    }
                    const uint32_t pos = swz(row, byte0 + piece * 16, 128);
                    *reinterpret_cast<uint4*>(stg + pos) = oh;
                    if constexpr (C::kSplit) *reinterpret_cast<uint4*>(stg + kTileBytes + pos) = ol;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> the bulk copy
        epi_bar_sync();
        if (store_thread) {
            const int64_t at = (int64_t(rt) * sg.rt_chunks[buf] + tk.out_pos + ch) * kTileBytes;
            if (rows == 128) {
                bulk_s2g(sg.rt_hi[buf] + at, smem_u32(stg), kTileBytes);
                if constexpr (C::kSplit) bulk_s2g(sg.rt_lo[buf] + at, smem_u32(stg + kTileBytes), kTileBytes);
            } else {  // the leading rows of each K-half
                for (int hf = 0; hf < 2; ++hf) {
                    const uint32_t o = uint32_t(hf) * (kTileBytes / 2);
                    bulk_s2g(sg.rt_hi[buf] + at + o, smem_u32(stg + o), uint32_t(rows) * 64u);
                    if constexpr (C::kSplit)
                        bulk_s2g(sg.rt_lo[buf] + at + o, smem_u32(stg + kTileBytes + o), uint32_t(rows) * 64u);
                }
            }
            bulk_commit();
        }
    }
}

// A generator lane's row: its point pre-scaled by -2, with 1 in the norm's
// slot, so that |y|^2 - 2 x.y is one FMA chain over the column point's DP
// floats (coordinates, then |y|^2, then zeros); n = |x|^2.  Cached across
// the stages of a task piece (rows, segment, row block).
template <int DP>
struct GenRow {
    float x[DP];
    float n;
    int64_t rows;
    int seg, rb;
};
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// The segment's generator constants, read once per job.
struct GenConst {
    const float4* tab;  // point table
    float scale;        // Gaussian: -inv log2(e); IMQ: inv
    float shift;
    int dim;
};
// The items of one generated stage that warp gw owns: item i = (block rb of
// 32 rows, 16-byte column group g), i = gw, gw + kGenWarps, ...; lane = row
// rb * 32 + lane.  DP: floats per point, GAUSS: the kernel (compile time).
// Entries: d2 = max(|x|^2 + |y|^2 - 2 x.y, 0) (exactly 0 for the same
// index); Gaussian exp(-d2 inv) = 2^(d2 * (-inv log2 e)); IMQ
// 1 / sqrt(1 + d2 inv); plus the shift on the same index (K_ii).  Written
// in the MMA layout.
template <int MODE, int DP, bool GAUSS>
__device__ __forceinline__ void gen_stage(GenRow<DP>& R, const GenJob& jb, const GenConst& gc, const float* cpts,
                                          uint8_t* bh, uint8_t* bl, int gw, int lane) {
    constexpr bool kSplit = MODE == TC_BF16X3;
    constexpr int kPer = MODE == TC_TF32 ? 4 : 8;         // columns per 16-byte group
    constexpr int kGroups = 4 * (kSplit ? 1 : 2);         // 16-byte column groups per stage
    const int nrb = (jb.n_pad + 31) / 32;
    const float scale = gc.scale;
    const float4* tab = gc.tab;
    for (int item = gw; item < nrb * kGroups; item += kGenWarps) {
        const int rb = item % nrb, g = item / nrb;
        const int n = rb * 32 + lane;
        if (R.rows != jb.rows || R.seg != jb.seg || R.rb != rb) {
            float x[DP];
#pragma unroll
            for (int q4 = 0; q4 < DP / 4; ++q4) {
                float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
                if (n < jb.m) t = tab[(jb.rows + n) * (DP / 4) + q4];
                x[4 * q4] = t.x;
                x[4 * q4 + 1] = t.y;
                x[4 * q4 + 2] = t.z;
                x[4 * q4 + 3] = t.w;
            }
            R.n = 0.f;
#pragma unroll
            for (int d = 0; d < DP; ++d) {
                if (d == gc.dim) R.n = x[d];
                R.x[d] = d == gc.dim ? 1.f : -2.f * x[d];
            }
            R.rows = jb.rows;
            R.seg = jb.seg;
            R.rb = rb;
        }
        if (n >= jb.n_pad) continue;
        const int k0 = g * kPer;
        // entry e is on the diagonal (the same index-list position) iff e == de
        const int64_t dd = jb.rows + n - (jb.cols + k0);
        const int de = dd >= 0 && dd < kPer ? int(dd) : -1;
        const int kv = n < jb.m ? jb.kvalid - k0 : 0;  // valid columns of this group (<= 0: none)
        // the kPer dot products advance together (independent FMA chains);
        // column points are read by the whole warp at one address
        const float4* cp = reinterpret_cast<const float4*>(cpts + k0 * DP);
        float v[kPer];
#pragma unroll
        for (int e = 0; e < kPer; ++e) v[e] = R.n;
#pragma unroll
        for (int q4 = 0; q4 < DP / 4; ++q4) {
#pragma unroll
            for (int e = 0; e < kPer; ++e) {
                const float4 c = cp[e * (DP / 4) + q4];
                v[e] = fmaf(R.x[4 * q4], c.x, v[e]);
                v[e] = fmaf(R.x[4 * q4 + 1], c.y, v[e]);
                v[e] = fmaf(R.x[4 * q4 + 2], c.z, v[e]);
                v[e] = fmaf(R.x[4 * q4 + 3], c.w, v[e]);
            }
        }
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
            const float d2 = e == de ? 0.f : fmaxf(v[e], 0.f);
            float y;
            if constexpr (GAUSS) y = ex2_approx(d2 * scale);
            else y = rsqrtf(fmaf(d2, scale, 1.f));
            if (e == de) y += gc.shift;
            v[e] = e < kv ? y : 0.f;
        }
        // group g of the stage: K-half g / 4, 16-byte group g % 4 of it
        const uint32_t pos = uint32_t(g >> 2) * uint32_t(jb.n_pad) * 64u + swz64(uint32_t(n), uint32_t((g & 3) * 16));
        if constexpr (MODE == TC_TF32) {
            *reinterpret_cast<float4*>(bh + pos) =
                make_float4(round_tf32(v[0]), round_tf32(v[1]), round_tf32(v[2]), round_tf32(v[3]));
        } else {
            uint4 oh, ol;
            __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(&oh);
            __nv_bfloat162* ll = reinterpret_cast<__nv_bfloat162*>(&ol);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                hh[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
                const float2 hf = __bfloat1622float2(hh[e]);
                ll[e] = __floats2bfloat162_rn(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
            }
            *reinterpret_cast<uint4*>(bh + pos) = oh;
            if constexpr (kSplit) *reinterpret_cast<uint4*>(bl + pos) = ol;
        }
    }
}

// The job loop of a generator warp for segments of point width DP: waits
// for each job (bounded), generates its share of the stage, publishes it.
// Returns the width of a job of another width (not consumed), or -1 at the
// stop job or on an error.  gbars: the job-full, job-empty and stage-done
// barriers, kStages each.
template <int MODE, int NMAX, int DP>
__device__ __noinline__ int gen_loop(const TcParams& p, const GenJob* jobs, const float* colring, uint8_t* base,
                                     uint64_t* gbars, int& seq, int gw, int lane) {
    using C = KCfg<MODE, NMAX, true>;
    GenRow<DP> R;
    R.rows = -1;
    R.seg = R.rb = -1;
    R.n = 0.f;
#pragma unroll
    for (int d = 0; d < DP; ++d) R.x[d] = 0.f;
    for (;; ++seq) {
        const int j = seq % C::kStages;
        const uint32_t full = smem_u32(&gbars[j]), empty = smem_u32(&gbars[C::kStages + j]);
        const uint32_t par = uint32_t((seq / C::kStages) & 1);
        bool ok = true;
        if (lane == 0) ok = mbar_wait(full, par, p.err, kErrGenerator);
        ok = __shfl_sync(0xffffffffu, ok, 0) != 0;  // lane 0 waited for the whole warp
        if (!ok) return -1;
        // every lane observes the completed phase itself (the job's fields
        // and the bulk-copied column points become visible)
        (void)mbar_try_wait(full, par);
        __syncwarp();
        const GenJob jb = jobs[j];
        if (jb.stop) return -1;
        const TcSeg& sg = p.segs[jb.seg];
        if (sg.dpad != DP) return sg.dpad;
        uint8_t* bh = base + jb.stage * C::kStageBytes + C::kW * C::kAUnit;
        uint8_t* bl = bh + C::kPart;  // split BF16x3: the lo copy of the stage
        const bool gauss = sg.gen_kind == GOFMM_GEN_GAUSSIAN;
        GenConst gc;
        gc.tab = reinterpret_cast<const float4*>(sg.pts);
        gc.scale = gauss ? -sg.gen_inv * 1.4426950408889634f : sg.gen_inv;  // log2(e)
        gc.shift = sg.gen_shift;
        gc.dim = sg.dim;
        const float* cpts = colring + j * (C::kColSlot / 4);
        if (gauss) gen_stage<MODE, DP, true>(R, jb, gc, cpts, bh, bl, gw, lane);
        else gen_stage<MODE, DP, false>(R, jb, gc, cpts, bh, bl, gw, lane);
        // generic writes -> visible to the MMAs (async proxy); this warp is
        // done with the job's column points
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(smem_u32(&gbars[2 * C::kStages + jb.stage]));  // stage written
            mbar_arrive(empty);
        }
    }
}

// Persistent grouped GEMM: CTA b processes tiles b, b + gridDim.x, ... (tile
// = task * n_rtiles + r-tile; tasks are sorted heaviest first).  The stage
// ring runs on across tiles and the accumulator is double-buffered in TMEM
// (2 x 256 columns), so the epilogue of one tile overlaps the MMAs of the
// next.
template <int MODE, int NMAX, bool GEN>
__global__ void __launch_bounds__(GEN ? kGenThreads : 192, 1) tc_gemm_kernel(const __grid_constant__ TcParams p) {
    using C = KCfg<MODE, NMAX, GEN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + C::kStages * C::kStageBytes);
    // generation (GEN): job ring from the producer to the generator warps,
    // per-stage "block tile written" barriers, per-stage generated flags
    uint8_t* gen_area = base + C::kStages * C::kStageBytes + 256;
    uint64_t* gbars = reinterpret_cast<uint64_t*>(gen_area);
    uint8_t* stage_isgen = gen_area + 3 * 8 * C::kStages;
    GenJob* jobs = reinterpret_cast<GenJob*>(gen_area + 256);
    float* colring = reinterpret_cast<float*>(gen_area + 1024);  // kStages slots of C::kColSlot bytes
    auto genq_full = [&](int j) { return smem_u32(&gbars[j]); };
    auto genq_empty = [&](int j) { return smem_u32(&gbars[C::kStages + j]); };
    auto gen_done = [&](int s) { return smem_u32(&gbars[2 * C::kStages + s]); };
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * C::kStages + 9);
    int* tid_slot = reinterpret_cast<int*>(tmem_slot + 1);  // [2]: tile ids handed from producer to consumers
    const uint32_t s_base = smem_u32(base);
    auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
    auto empty_bar = [&](int s) { return smem_u32(&bars[C::kStages + s]); };
    auto tfull_bar = [&](int a) { return smem_u32(&bars[2 * C::kStages + a]); };
    auto tempty_bar = [&](int a) { return smem_u32(&bars[2 * C::kStages + 2 + a]); };
    const uint32_t drain_bar = smem_u32(&bars[2 * C::kStages + 4]);
    auto idfull_bar = [&](int a) { return smem_u32(&bars[2 * C::kStages + 5 + a]); };
    auto idempty_bar = [&](int a) { return smem_u32(&bars[2 * C::kStages + 7 + a]); };
    // dynamic tile claiming from a counter (with dependency waits where the
    // segments carry dependency arrays), else a static round-robin split
    const bool dyn = p.tile_next != nullptr;
    // stage s: A0_hi .. A(kW-1)_hi | B_hi | (A0_lo .. | B_lo): kSub K-halves of
    // the right-hand-side tiles of r-tiles rt .. rt + kW - 1 and of the block tile
    auto sA = [&](int s, int lo, int w) { return s_base + s * C::kStageBytes + lo * C::kPart + w * C::kAUnit; };
    auto sB = [&](int s, int lo) { return s_base + s * C::kStageBytes + lo * C::kPart + C::kW * C::kAUnit; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = p.ntiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::kStages; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull_bar(a), 1);
            mbar_init(tempty_bar(a), 4);  // one arrival per epilogue warp
        }
        mbar_init(drain_bar, 1);
        for (int a = 0; a < 2; ++a) {
            mbar_init(idfull_bar(a), 1);
            mbar_init(idempty_bar(a), 5);  // MMA thread + four epilogue warps
        }
        if constexpr (GEN) {
            for (int j = 0; j < C::kStages; ++j) {
                mbar_init(genq_full(j), 1);        // the producer posts a job
                mbar_init(genq_empty(j), kGenWarps);  // every generator warp is done with it
                mbar_init(gen_done(j), kGenWarps);    // every generator warp wrote its part of the stage
            }
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(C::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer: stream the operand stages of every tile of this CTA
            int stage = 0, issued = 0, gseq = 0;
            uint32_t phase = 0;
            bool ok = true;
            bool list_left = true;  // ready queue: the list still has tiles
            for (int i = 0, t = blockIdx.x; ok; ++i) {
                if (dyn) {
                    // take the next tile in priority order (or from the ready
                    // queue) and hand its id on
                    if (!mbar_wait(idempty_bar(i & 1), uint32_t(((i >> 1) & 1) ^ 1), p.err, kErrProducer)) break;
                    if (p.ready.queue) {
                        const int c = ready_claim(p, list_left);
                        t = c < 0 ? ntiles : c;
                    } else {
                        t = atomicAdd(p.tile_next, 1);
                    }
                    tid_slot[i & 1] = t < ntiles ? t : -1;
                    mbar_arrive(idfull_bar(i & 1));
                } else if (i > 0) {
                    t += gridDim.x;
                }
                if (t >= ntiles) break;
                const TcTile tt = fetch_tile(p, t);
                const TcSeg& sg = p.segs[tt.seg];
                const TcTask tk = sg.tasks[tt.task];
                const int rt = tt.rt;
                const int nw = tile_width(tt);
                const uint32_t b_half = uint32_t(tk.n_pad) * 64u;  // one K-half of a block chunk tile
                uint32_t a_stage = 0;  // right-hand-side bytes of one stage (hi or lo part)
                for (int w = 0; w < nw; ++w) a_stage += uint32_t(C::kSub * rt_rows(sg.r, rt + w)) * 64u;
                if (dyn && sg.dep_off) {
                    // results of other tiles of this launch the task needs
                    // before it starts (the operands are waited for slab by slab)
                    for (int d = sg.dep_off[tt.task]; d < sg.dep_off[tt.task + 1] && ok; ++d)
                        for (int w = 0; w < nw && ok; ++w)
                            ok = wait_counter(sg.counters + int64_t(sg.deps[2 * d]) * sg.dep_nrt + rt + w,
                                              sg.deps[2 * d + 1], p.err);
                    if (!ok) break;
                }
                for (int si = tk.slab0; si < tk.slab1 && ok; ++si) {
                    const TcSlab sl = sg.slabs[si];
                    if (dyn && sg.dep_off) {
                        // this slab's right-hand sides, written earlier in the
                        // launch by other tiles: wait (bounded), then make the
                        // generic writes visible to the bulk copies
                        for (int w = 0; w < nw && ok; ++w) {
                            if (sl.dep_c0 >= 0)
                                ok = wait_counter(sg.counters + int64_t(sl.dep_c0) * sg.dep_nrt + rt + w, sl.dep_n0,
                                                  p.err);
                            if (ok && sl.dep_c1 >= 0)
                                ok = wait_counter(sg.counters + int64_t(sl.dep_c1) * sg.dep_nrt + rt + w, sl.dep_n1,
                                                  p.err);
                        }
                        if (!ok) break;
                        asm volatile("fence.proxy.async.global;" ::: "memory");
                    }
                    if constexpr (!GEN) {
                        if (sl.gen) {  // the host launches the generator variant for these; never read as tiles
                            atomicCAS(p.err, 0, kErrGenerator);
                            ok = false;
                            break;
                        }
                    }
                    // r-tile rt + w of the slab's right-hand sides: a_hi + w * a_rt
                    const int64_t a_off = (int64_t(rt) * sg.rt_chunks[sl.a_buf] + sl.a_chunk0) * kTileBytes;
                    const int64_t a_rt = int64_t(sg.rt_chunks[sl.a_buf]) * kTileBytes;
                    const uint8_t* a_hi = sg.rt_hi[sl.a_buf] + a_off;
                    const uint8_t* a_lo = C::kSplit ? sg.rt_lo[sl.a_buf] + a_off : nullptr;
                    const bool gen = GEN && sl.gen;  // block tiles written by the generator warps
                    const uint32_t b_stage = gen ? 0u : uint32_t(C::kSub) * b_half;
                    for (int q = 0; q < 2 * sl.nchunks / C::kSub; ++q) {
                        if (!mbar_wait(empty_bar(stage), phase ^ 1u, p.err, kErrProducer)) { ok = false; break; }
                        if constexpr (GEN) {
                            stage_isgen[stage] = gen ? 1 : 0;
                            if (gen) {
                                const int j = gseq % C::kStages;
                                if (!mbar_wait(genq_empty(j), uint32_t(((gseq / C::kStages) & 1) ^ 1), p.err,
                                               kErrProducer)) { ok = false; break; }
                                GenJob& jb = jobs[j];
                                jb.rows = sl.b_off;
                                jb.cols = sl.gen_cols + int64_t(q) * C::kStageK;
                                jb.seg = tt.seg;
                                jb.stage = stage;
                                jb.m = tk.m;
                                jb.kvalid = max(0, min(C::kStageK, sl.k - q * C::kStageK));
                                jb.n_pad = tk.n_pad;
                                jb.stop = 0;
                                // the stage's column points (consecutive rows of the
                                // point table, dpad floats each: a multiple of 16
                                // bytes) into the job's slot
                                const uint32_t cbytes = uint32_t(jb.kvalid) * uint32_t(sg.dpad) * 4u;
                                if (cbytes) {
                                    mbar_expect_tx(genq_full(j), cbytes);
                                    bulk_g2s(smem_u32(colring) + uint32_t(j * C::kColSlot),
                                             sg.pts + jb.cols * sg.dpad, cbytes, genq_full(j));
                                } else {
                                    mbar_arrive(genq_full(j));
                                }
                                ++gseq;
                            }
                        }
                        // stage q: K-halves [q kSub, (q + 1) kSub) of the slab's chunks
                        const int64_t ah = int64_t(q) * C::kAUnit;
                        const int64_t bh = int64_t(q) * b_stage;
                        // r-tiles past r / 16 rows: only their leading rows (rt_rows)
                        mbar_expect_tx(full_bar(stage), (C::kSplit ? 2u : 1u) * (a_stage + b_stage));
                        for (int w = 0; w < nw; ++w) {
                            const uint32_t ab = uint32_t(rt_rows(sg.r, rt + w)) * 64u;
                            if (ab == 128u * 64u) {
                                bulk_g2s(sA(stage, 0, w), a_hi + w * a_rt + ah, C::kAUnit, full_bar(stage));
                                if constexpr (C::kSplit)
                                    bulk_g2s(sA(stage, 1, w), a_lo + w * a_rt + ah, C::kAUnit, full_bar(stage));
                                continue;
                            }
#pragma unroll
                            for (int hs = 0; hs < C::kSub; ++hs) {
                                bulk_g2s(sA(stage, 0, w) + hs * C::kHalfA, a_hi + w * a_rt + ah + hs * C::kHalfA, ab,
                                         full_bar(stage));
                                if constexpr (C::kSplit)
                                    bulk_g2s(sA(stage, 1, w) + hs * C::kHalfA, a_lo + w * a_rt + ah + hs * C::kHalfA,
                                             ab, full_bar(stage));
                            }
                        }
                        if (!gen) {
                            bulk_g2s(sB(stage, 0), sg.b_hi + sl.b_off + bh, b_stage, full_bar(stage));
                            if constexpr (C::kSplit)
                                bulk_g2s(sB(stage, 1), sg.b_lo + sl.b_off + bh, b_stage, full_bar(stage));
                        }
                        ++issued;
                        if (++stage == C::kStages) { stage = 0; phase ^= 1u; }
                    }
                }
            }
            if constexpr (GEN) {
                // release the generator warps (bounded: they may have stopped on an error)
                const int j = gseq % C::kStages;
                if (mbar_wait(genq_empty(j), uint32_t(((gseq / C::kStages) & 1) ^ 1), p.err, kErrProducer)) {
                    jobs[j].stop = 1;
                    mbar_arrive(genq_full(j));
                }
            }
            if (!ok) {
                // drain: wait (bounded) for the copies of the last issued stages
                const int outstanding = issued < C::kStages ? issued : C::kStages;
                for (int q = 1; q <= outstanding; ++q) {
                    const int idx = issued - q;
                    const long long t0 = clock64();
                    while (!mbar_try_wait(full_bar(idx % C::kStages), uint32_t((idx / C::kStages) & 1)) &&
                           clock64() - t0 < kSpinLimit) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer (one thread).  Accumulator buffers: a one-r-tile
            // tile takes the next of the two in turn, a two-r-tile tile both.
            int stage = 0, i = 0, bnext = 0;
            uint32_t fills = 0;  // bit b: parity of the fills of accumulator buffer b
            uint32_t phase = 0, genpar = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok; t += gridDim.x, ++i) {
                if (dyn) {
                    if (!mbar_wait(idfull_bar(i & 1), uint32_t((i >> 1) & 1), p.err, kErrMma)) break;
                    t = tid_slot[i & 1];
                    mbar_arrive(idempty_bar(i & 1));
                    if (t < 0) break;
                }
                if (t >= ntiles) break;
                const TcTile tt = fetch_tile(p, t);
                const TcTask tk = p.segs[tt.seg].tasks[tt.task];
                const int nw = tile_width(tt);
                const int nb = acc_buffers(nw, tk.n_pad);
                const int b0 = nb == 2 ? 0 : bnext;
                if (nb == 1) bnext ^= 1;
                for (int b = 0; b < nb && ok; ++b)
                    ok = mbar_wait(tempty_bar(b0 + b), ((fills >> (b0 + b)) & 1u) ^ 1u, p.err, kErrMma);
                if (!ok) break;
                tc_fence_after();
                const uint32_t tacc = tmem + uint32_t(b0 * kAccBufCols);  // r-tile rt + w: tacc + w * acc_step
                const uint32_t acc_step = uint32_t(acc_stride(nw, nb));
                const bool rowf = row_form(tk, nw, C::kSplit);
                const uint32_t idesc = make_idesc(MODE == TC_TF32 ? 2 : 1, rowf ? 2 * 128 : tk.n_pad);
                const uint32_t b_half = uint32_t(tk.n_pad) * 64u;
                for (int q = 0; q < 2 * tk.nchunks / C::kSub; ++q) {
                    if (!mbar_wait(full_bar(stage), phase, p.err, kErrMma)) { ok = false; break; }
                    if constexpr (GEN) {
                        if (stage_isgen[stage]) {  // block tile written by the generator warps
                            if (!mbar_wait(gen_done(stage), (genpar >> stage) & 1u, p.err, kErrMma)) {
                                ok = false;
                                break;
                            }
                            genpar ^= 1u << stage;
                        }
                    }
                    tc_fence_after();
                    // one descriptor per stage; the operands' descriptors differ
                    // from it by their shared-memory offsets (in 16-byte units)
                    const uint64_t d0 = sw64_desc(sA(stage, 0, 0));
                    if constexpr (C::kSplit) {
                        if (rowf) {  // block (M = 128) x both r-tiles (N = 256), hi.hi + lo.hi + hi.lo
                            constexpr uint64_t lo = uint64_t(C::kPart >> 4);
                            const uint64_t dk = d0 + (uint32_t(C::kW * C::kAUnit) >> 4);
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                const uint64_t off = uint64_t(kk * 2);
                                mma<MODE>(tacc, dk + off, d0 + off, idesc, (q > 0 || kk > 0) ? 1u : 0u);
                                mma<MODE>(tacc, dk + lo + off, d0 + off, idesc, 1u);
                                mma<MODE>(tacc, dk + off, d0 + lo + off, idesc, 1u);
                            }
                            mma_commit(empty_bar(stage));
                            if (++stage == C::kStages) { stage = 0; phase ^= 1u; }
                            continue;
                        }
                    }
#pragma unroll
                    for (int hs = 0; hs < C::kSub; ++hs) {
                        const uint64_t db = d0 + (uint32_t(C::kW * C::kAUnit + hs * b_half) >> 4);
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint64_t off = uint64_t(kk * 2);  // 32 bytes per MMA K step
                            const uint32_t acc_in = (q > 0 || hs > 0 || kk > 0) ? 1u : 0u;
#pragma unroll
                            for (int w = 0; w < C::kW; ++w) {
                                if (w < nw) {
                                    const uint64_t da = d0 + uint64_t((w * C::kAUnit + hs * C::kHalfA) >> 4) + off;
                                    const uint32_t tw = tacc + uint32_t(w) * acc_step;
                                    mma<MODE>(tw, da, db + off, idesc, acc_in);
                                    if constexpr (C::kSplit) {
                                        constexpr uint64_t lo = uint64_t(C::kPart >> 4);
                                        mma<MODE>(tw, da, db + lo + off, idesc, 1u);
                                        mma<MODE>(tw, da + lo, db + off, idesc, 1u);
                                    }
                                }
                            }
                        }
                    }
                    mma_commit(empty_bar(stage));
                    if (++stage == C::kStages) { stage = 0; phase ^= 1u; }
                }
                for (int b = 0; b < nb; ++b) {
                    mma_commit(tfull_bar(b0 + b));
                    fills ^= 1u << (b0 + b);
                }
            }
            // no MMA may still be running when TMEM is freed
            mma_commit(drain_bar);
            const long long t0 = clock64();
            while (!mbar_try_wait(drain_bar, 0) && clock64() - t0 < kSpinLimit) {
            }
        }
    } else if (warp < 6) {
        // ---- epilogue: warps 2..5 own TMEM lane quarters (warp % 4)
        const int q4 = warp & 3;
        const int row = q4 * 32 + lane;  // row of the MMA tile = column of r
        const bool store_thread = warp == 2 && lane == 0;  // issues the staged tiles' bulk stores
        uint8_t* stg = base + C::kStages * C::kStageBytes + 256;  // staging tile (kernels without generator warps)
        int i = 0, bnext = 0;
        uint32_t fills = 0;  // the MMA issuer's buffer sequence, replayed
        for (int t = blockIdx.x;; t += gridDim.x, ++i) {
            if (dyn) {
                bool okid = mbar_wait(idfull_bar(i & 1), uint32_t((i >> 1) & 1), p.err, kErrEpilogue);
                okid = epi_bar_and(okid) != 0;  // the four warps leave together (they share barrier 2)
                if (!okid) break;
                t = tid_slot[i & 1];
                __syncwarp();
                if (lane == 0) mbar_arrive(idempty_bar(i & 1));
                if (t < 0) break;
            }
            if (t >= ntiles) break;
            const TcTile tt = fetch_tile(p, t);
            const TcSeg& sg = p.segs[tt.seg];
            const TcTask tk = sg.tasks[tt.task];
            const int rt = tt.rt;
            const int nw = tile_width(tt);
            const int nb = acc_buffers(nw, tk.n_pad);
            const int b0 = nb == 2 ? 0 : bnext;
            if (nb == 1) bnext ^= 1;
            const int acc_step = acc_stride(nw, nb);
            const int per_buf = nb == 2 ? nw / 2 : nw;  // accumulators in one buffer
            if (tk.accumulate && tk.out_kind != OUT_U) {
                // an accumulating right-hand-side output adds to rows written
                // long before: bring this thread's part of them into L2 while
                // the MMAs run, so the read-modify-write below waits on L2,
                // not DRAM, once per 32 rows (the plans built here have no
                // such task: the downward pass pulls, see build_tc_plan)
                const int buf = tk.out_kind == OUT_WTIL ? 1 : 2;
                for (int w = 0; w < nw; ++w) {
                    if ((rt + w) * 128 + row >= sg.r) break;
                    for (int c = 0; c * C::kKc < tk.n_pad; ++c) {
                        const int64_t off = (int64_t(rt + w) * sg.rt_chunks[buf] + tk.out_pos + c) * kTileBytes;
                        prefetch_l2(sg.rt_hi[buf] + off + swz(row, 0, 128));
                        prefetch_l2(sg.rt_hi[buf] + off + swz(row, 64, 128));
                        if constexpr (C::kSplit) {
                            prefetch_l2(sg.rt_lo[buf] + off + swz(row, 0, 128));
                            prefetch_l2(sg.rt_lo[buf] + off + swz(row, 64, 128));
                        }
                    }
                }
            }
            bool ok = true;
            for (int b = 0; b < nb && ok; ++b)
                ok = mbar_wait(tfull_bar(b0 + b), (fills >> (b0 + b)) & 1u, p.err, kErrEpilogue);
            // tcgen05.ld below is warp-collective, and the four warps share
            // barrier 2 (staged stores): all of them go on or none
            ok = epi_bar_and(ok) != 0;
            if (!ok) break;
            tc_fence_after();
            // RT outputs write the whole output segment of the task (zeros in the
            // padding columns and in rows r .. rt_rows), so every RT element a
            // later stage reads was written earlier in the same evaluation; only
            // accumulating outputs touch valid elements alone.
            const bool staged = !GEN && tk.out_kind != OUT_U && !tk.accumulate;
            if (row_form(tk, nw, C::kSplit)) {
                write_rows(sg, tk, rt, row, tmem + uint32_t(b0 * kAccBufCols) + (uint32_t(q4 * 32) << 16));
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty_bar(b0));
                fills ^= 1u << b0;
            }
            for (int w = 0; w < nw && !row_form(tk, nw, C::kSplit); ++w) {
                const uint32_t taddr = tmem + uint32_t(b0 * kAccBufCols + w * acc_step) + (uint32_t(q4 * 32) << 16);
                if (staged)
                    write_tile_staged<MODE>(sg, tk, rt + w, row, taddr, stg, store_thread);
                else
                    write_tile<MODE>(sg, tk, rt + w, row, taddr);
                // an accumulator buffer is free for the MMAs of a later tile as
                // soon as this tile's accumulators in it are read (a tile with
                // two buffers frees the first before draining the second)
                if ((w + 1) % per_buf == 0) {
                    const int b = w / per_buf;
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty_bar(b0 + b));
                    fills ^= 1u << (b0 + b);
                }
            }
            if (dyn && sg.sig) {
                // publish this warp's 32 rows of the tile: consumers wait for
                // four arrivals (one per epilogue warp) per task piece
                const int s0 = sg.sig[2 * tt.task], s1 = sg.sig[2 * tt.task + 1];
                if (s0 >= 0 || s1 >= 0) {
                    if (staged) {
                        // the bulk stores of the tile performed before any warp publishes
                        if (store_thread) bulk_wait_all();
                        epi_bar_sync();
                    }
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) {
                        __threadfence();
                        for (int w = 0; w < nw; ++w)
                            for (int c : {s0, s1}) {
                                if (c < 0) continue;
                                const int old = atomicAdd(sg.counters + int64_t(c) * sg.dep_nrt + rt + w, 1);
                                // the final arrival releases the queued tiles waiting on it
                                if (p.ready.queue && old + 1 == p.ready.req[c]) ready_release(p, c * sg.dep_nrt + rt + w);
                            }
                    }
                }
            }
        }
        if (store_thread) bulk_wait_all();  // no bulk store may still read the staging tile
    } else {
        if constexpr (GEN) {
            // ---- generator warps 6..: block tiles of generated slabs,
            // written into the stage's B region in the MMA layout.  The job
            // loop runs in the instantiation for the point width of the
            // current segment and returns here when a job of another width
            // arrives (a batch can mix matrices) or at the end.
            int seq = 0, dpad = 0;
            for (;;) {
                if (dpad == 0) {  // width of the next job, once it is posted
                    const int j = seq % C::kStages;
                    const uint32_t par = uint32_t((seq / C::kStages) & 1);
                    bool ok = true;
                    if (lane == 0) ok = mbar_wait(genq_full(j), par, p.err, kErrGenerator);
                    ok = __shfl_sync(0xffffffffu, ok, 0) != 0;
                    if (!ok) break;
                    (void)mbar_try_wait(genq_full(j), par);
                    __syncwarp();
                    if (jobs[j].stop) break;
                    dpad = p.segs[jobs[j].seg].dpad;
                }
                switch (dpad) {  // the host allows 4, 8, 12 or 16 floats per point
                    case 4: dpad = gen_loop<MODE, NMAX, 4>(p, jobs, colring, base, gbars, seq, warp - 6, lane); break;
                    case 8: dpad = gen_loop<MODE, NMAX, 8>(p, jobs, colring, base, gbars, seq, warp - 6, lane); break;
                    case 12: dpad = gen_loop<MODE, NMAX, 12>(p, jobs, colring, base, gbars, seq, warp - 6, lane); break;
                    default: dpad = gen_loop<MODE, NMAX, 16>(p, jobs, colring, base, gbars, seq, warp - 6, lane); break;
                }
                if (dpad < 0) break;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// SM-pair variant (tcgen05 cta_group::2).  A cluster of two CTAs computes one
// 256 x N output tile: two r-tiles (2q and 2q + 1) of one task.  CTA c of the
// pair stages the 128 right-hand-side columns of r-tile 2q + c and block rows
// [c N/2, (c + 1) N/2) of each chunk; the even CTA issues the M = 256 MMAs,
// which read both CTAs' shared memory and leave each CTA's 128 accumulator
// rows in that CTA's TMEM, so each CTA's epilogue writes its own r-tile as in
// the single-SM kernel.  Per SM, a chunk then stages 128 + N/2 rows instead
// of 128 + N for the same MMA work.
//
// Bulk copies signal a barrier of their own CTA only, so the odd CTA's MMA
// warp (idle otherwise) forwards each completed stage to the even CTA's
// barrier with a remote arrive; the even CTA's commits arrive on both CTAs'
// barriers (multicast).  Static tile order (the staged schedule).
template <int MODE, int NMAX>
struct Cfg2 {
    static constexpr bool kSplit = MODE == TC_BF16X3;
    static constexpr int kBHalf = NMAX / 2 * 128;  // bytes of one CTA's half block tile
    static constexpr int kBQuarter = NMAX / 2 * 64;  // ... of one K-half of it
    static constexpr int kStageBytes = (kSplit ? 2 : 1) * (kTileBytes + kBHalf);
    static constexpr int kStages = (200 * 1024 / kStageBytes) < 8 ? (200 * 1024 / kStageBytes) : 8;
    static constexpr int kSmem = kStages * kStageBytes + 1024 + 256;
    static constexpr int kTmemCols = 2 * NMAX;  // two accumulators
    static_assert(kStages >= 2 && kSmem <= 227 * 1024, "stage ring");
};

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// shared::cluster address of the same shared-memory offset in CTA `rank`
__device__ __forceinline__ uint32_t peer_addr(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait with cluster-scope acquire (arrivals from the other CTA).
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, int* err, int code) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if (it % kPollsPerCheck == 0) {
            if (*reinterpret_cast<volatile int*>(err) != 0) return false;
            if (clock64() - t0 > kSpinLimit) {
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t cluster_addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(cluster_addr) : "memory");
    return v;
}
template <int MODE>
__device__ __forceinline__ void mma_pair(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    if constexpr (MODE == TC_TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
    }
}
// commit of the pair's MMAs issued so far: one arrival on the barrier at the
// same offset in both CTAs
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            bar),
        "h"(uint16_t(3))
        : "memory");
}

template <int MODE, int NMAX>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(192, 1)
    tc_gemm_pair_kernel(const __grid_constant__ TcParams p) {
    using C = Cfg2<MODE, NMAX>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + C::kStages * C::kStageBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * C::kStages + 5);
    const uint32_t s_base = smem_u32(base);
    auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
    auto empty_bar = [&](int s) { return smem_u32(&bars[C::kStages + s]); };
    auto tfull_bar = [&](int a) { return smem_u32(&bars[2 * C::kStages + a]); };
    auto tempty_bar = [&](int a) { return smem_u32(&bars[2 * C::kStages + 2 + a]); };
    const uint32_t drain_bar = smem_u32(&bars[2 * C::kStages + 4]);
    // stage s: A_hi | B_hi half | (A_lo | B_lo half)
    auto sA = [&](int s, int lo) { return s_base + s * C::kStageBytes + lo * (kTileBytes + C::kBHalf); };
    auto sB = [&](int s, int lo) { return sA(s, lo) + kTileBytes; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t crank = cluster_rank();
    const bool leader = crank == 0;
    const int pair = int(blockIdx.x >> 1), npairs = int(gridDim.x >> 1);
    const int ntiles = p.ntiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::kStages; ++s) {
            mbar_init(full_bar(s), leader ? 2 : 1);  // leader: own copies + the odd CTA's forward
            mbar_init(empty_bar(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull_bar(a), 1);
            mbar_init(tempty_bar(a), 8);  // four epilogue warps in each CTA (used in the leader)
        }
        mbar_init(drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(C::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // barriers of both CTAs initialised, TMEM allocated
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // the two CTAs must address the same TMEM columns
    if (!leader && threadIdx.x == 0 && ld_cluster_u32(peer_addr(smem_u32(tmem_slot), 0)) != tmem)
        atomicCAS(p.err, 0, kErrTmemPair);
    cluster_sync_all();
    const bool run = *reinterpret_cast<volatile int*>(p.err) == 0;

    if (run && warp == 0) {
        if (lane == 0) {
            // ---- producer (both CTAs): own r-tile and own half of each block chunk
            int stage = 0, issued = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int t = pair; t < ntiles && ok; t += npairs) {
                const TcTile tt = fetch_tile(p, t);
                const TcSeg& sg = p.segs[tt.seg];
                const TcTask tk = sg.tasks[tt.task];
                const int rt = 2 * tt.rt + int(crank);
                const bool live = rt * 128 < sg.r;  // the odd half of the last pair may be padding
                const uint32_t half = uint32_t(tk.n_pad) / 2u * 128u;
                const uint32_t a_rows = uint32_t(rt_rows(sg.r, rt));  // leading rows of each K-half
                const uint32_t a_bytes = 2u * a_rows * 64u;
                for (int si = tk.slab0; si < tk.slab1 && ok; ++si) {
                    const TcSlab sl = sg.slabs[si];
                    if (sl.gen) {  // the pair schedule runs cached blocks only (the host refuses generated plans)
                        atomicCAS(p.err, 0, kErrGenerator);
                        ok = false;
                        break;
                    }
                    const int64_t a_off = (int64_t(rt) * sg.rt_chunks[sl.a_buf] + sl.a_chunk0) * kTileBytes;
                    const int64_t b_row = int64_t(tk.n_pad) * 128;  // one chunk tile
                    const uint32_t qrt = half / 2u;                 // this CTA's rows of one K-half
                    const int64_t b_off = sl.b_off + int64_t(crank) * qrt;
                    for (int c = 0; c < sl.nchunks; ++c) {
                        if (!mbar_wait(empty_bar(stage), phase ^ 1u, p.err, kErrProducer)) { ok = false; break; }
                        mbar_expect_tx(full_bar(stage), (C::kSplit ? 2u : 1u) * (a_bytes + half));
                        if (a_rows == 128)
                            bulk_g2s(sA(stage, 0), sg.rt_hi[sl.a_buf] + a_off + int64_t(c) * kTileBytes, kTileBytes,
                                     full_bar(stage));
                        else if (live)
                            for (int hf = 0; hf < 2; ++hf)
                                bulk_g2s(sA(stage, 0) + hf * (kTileBytes / 2),
                                         sg.rt_hi[sl.a_buf] + a_off + int64_t(c) * kTileBytes + hf * (kTileBytes / 2),
                                         a_rows * 64u, full_bar(stage));
                        for (int h = 0; h < 2; ++h)
                            bulk_g2s(sB(stage, 0) + h * C::kBQuarter, sg.b_hi + b_off + int64_t(c) * b_row + h * (b_row / 2),
                                     qrt, full_bar(stage));
                        if constexpr (C::kSplit) {
                            if (a_rows == 128)
                                bulk_g2s(sA(stage, 1), sg.rt_lo[sl.a_buf] + a_off + int64_t(c) * kTileBytes,
                                         kTileBytes, full_bar(stage));
                            else if (live)
                                for (int hf = 0; hf < 2; ++hf)
                                    bulk_g2s(sA(stage, 1) + hf * (kTileBytes / 2),
                                             sg.rt_lo[sl.a_buf] + a_off + int64_t(c) * kTileBytes +
                                                 hf * (kTileBytes / 2),
                                             a_rows * 64u, full_bar(stage));
                            for (int h = 0; h < 2; ++h)
                                bulk_g2s(sB(stage, 1) + h * C::kBQuarter,
                                         sg.b_lo + b_off + int64_t(c) * b_row + h * (b_row / 2), qrt, full_bar(stage));
                        }
                        ++issued;
                        if (++stage == C::kStages) { stage = 0; phase ^= 1u; }
                    }
                }
            }
            if (!ok) {
                const int outstanding = issued < C::kStages ? issued : C::kStages;
                for (int q = 1; q <= outstanding; ++q) {
                    const int idx = issued - q;
                    const long long t0 = clock64();
                    while (!mbar_try_wait(full_bar(idx % C::kStages), uint32_t((idx / C::kStages) & 1)) &&
                           clock64() - t0 < kSpinLimit) {
                    }
                }
            }
        }
    } else if (run && warp == 1) {
        if (lane == 0 && leader) {
            // ---- MMA issuer (even CTA, one thread)
            int stage = 0, i = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int t = pair; t < ntiles && ok; t += npairs, ++i) {
                const TcTile tt = fetch_tile(p, t);
                const TcTask tk = p.segs[tt.seg].tasks[tt.task];
                const int acc = i & 1;
                if (!mbar_wait_cluster(tempty_bar(acc), uint32_t(((i >> 1) & 1) ^ 1), p.err, kErrMma)) break;
                tc_fence_after();
                const uint32_t tacc = tmem + uint32_t(acc * NMAX);
                const uint32_t idesc = (1u << 4) | (uint32_t(MODE == TC_TF32 ? 2 : 1) << 7) |
                                       (uint32_t(MODE == TC_TF32 ? 2 : 1) << 10) | (uint32_t(tk.n_pad >> 3) << 17) |
                                       (uint32_t(256 >> 4) << 24);
                for (int q = 0; q < tk.nchunks; ++q) {
                    if (!mbar_wait_cluster(full_bar(stage), phase, p.err, kErrMma)) { ok = false; break; }
                    tc_fence_after();
#pragma unroll
                    for (int h = 0; h < 2; ++h) {  // the chunk's two K-halves
                        const uint64_t da = sw64_desc(sA(stage, 0) + h * (kTileBytes / 2));
                        const uint64_t db = sw64_desc(sB(stage, 0) + h * C::kBQuarter);
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint64_t off = uint64_t(kk * 2);
                            mma_pair<MODE>(tacc, da + off, db + off, idesc, (q > 0 || h > 0 || kk > 0) ? 1u : 0u);
                            if constexpr (C::kSplit) {
                                const uint64_t dal = sw64_desc(sA(stage, 1) + h * (kTileBytes / 2));
                                const uint64_t dbl = sw64_desc(sB(stage, 1) + h * C::kBQuarter);
                                mma_pair<MODE>(tacc, da + off, dbl + off, idesc, 1u);
                                mma_pair<MODE>(tacc, dal + off, db + off, idesc, 1u);
                            }
                        }
                    }
                    mma_commit_pair(empty_bar(stage));
                    if (++stage == C::kStages) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                mma_commit_pair(tfull_bar(acc));
            }
            asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             drain_bar)
                         : "memory");
            const long long t0 = clock64();
            while (!mbar_try_wait(drain_bar, 0) && clock64() - t0 < kSpinLimit) {
            }
        } else if (lane == 0) {
            // ---- odd CTA: forward each landed stage to the even CTA's barrier
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int t = pair; t < ntiles && ok; t += npairs) {
                const TcTile tt = fetch_tile(p, t);
                const TcTask tk = p.segs[tt.seg].tasks[tt.task];
                for (int q = 0; q < tk.nchunks; ++q) {
                    if (!mbar_wait(full_bar(stage), phase, p.err, kErrMma)) { ok = false; break; }
                    mbar_arrive_cluster(peer_addr(full_bar(stage), 0));
                    if (++stage == C::kStages) { stage = 0; phase ^= 1u; }
                }
            }
        }
    } else if (run) {
        // ---- epilogue: warps 2..5 own TMEM lane quarters (warp % 4)
        const int q4 = warp & 3;
        const int row = q4 * 32 + lane;
        const uint32_t tempty_leader = peer_addr(tempty_bar(0), 0);  // + 8 bytes for accumulator 1
        int i = 0;
        for (int t = pair; t < ntiles; t += npairs, ++i) {
            const TcTile tt = fetch_tile(p, t);
            const TcSeg& sg = p.segs[tt.seg];
            const TcTask tk = sg.tasks[tt.task];
            const int rt = 2 * tt.rt + int(crank);
            const int acc = i & 1;
            bool ok = mbar_wait_cluster(tfull_bar(acc), uint32_t((i >> 1) & 1), p.err, kErrEpilogue);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc_fence_after();
            const uint32_t taddr = tmem + uint32_t(acc * NMAX) + (uint32_t(q4 * 32) << 16);
            if (rt * 128 < sg.r) write_tile<MODE>(sg, tk, rt, row, taddr);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(tempty_leader + uint32_t(acc * 8));
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // no MMA of the pair runs and no TMEM read is pending
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kTmemCols)
                     : "memory");
    }
}

// W (original order, FP32) -> WT in RT layout, one 128 x KC tile per CTA.
template <int MODE>
__global__ void __launch_bounds__(256) tc_gather_kernel(const float* __restrict__ W, int64_t ldw,
                                                        const int64_t* __restrict__ perm,
                                                        const int64_t* __restrict__ chunk_pos,
                                                        const int32_t* __restrict__ chunk_valid, uint8_t* wt_hi,
                                                        uint8_t* wt_lo, int64_t wt_chunks, int r) {
    using C = Cfg<MODE>;
    __shared__ __align__(16) uint8_t hi[kTileBytes];
    __shared__ __align__(16) uint8_t lo[C::kSplit ? kTileBytes : 16];
    const int64_t c = blockIdx.x;
    const int rt = blockIdx.y;
    const int64_t pos = chunk_pos[c];
    const int valid = chunk_valid[c];
    const int rows = rt_rows(r, rt);  // the rows later copies read (zeros from r on)
    for (int e = threadIdx.x; e < rows * C::kKc; e += blockDim.x) {
        const int k = e / rows, jj = e % rows, j = rt * 128 + jj;
        float x = 0.f;
        if (k < valid && j < r) x = W[perm[pos + k] * ldw + j];
        const uint32_t at = swz(uint32_t(jj), uint32_t(k * C::kEs), 128);
        if constexpr (MODE == TC_TF32) {
            *reinterpret_cast<float*>(hi + at) = round_tf32(x);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            *reinterpret_cast<__nv_bfloat16*>(hi + at) = h;
            if constexpr (C::kSplit)
                *reinterpret_cast<__nv_bfloat16*>(lo + at) = __float2bfloat16_rn(x - __bfloat162float(h));
        }
    }
    __syncthreads();
    const int64_t off = (int64_t(rt) * wt_chunks + c) * kTileBytes;
    for (int e = threadIdx.x; e < kTileBytes / 16; e += blockDim.x) {
        if ((e % (kTileBytes / 32)) / 4 >= rows) continue;  // 16-byte group -> row of its K-half
        reinterpret_cast<uint4*>(wt_hi + off)[e] = reinterpret_cast<const uint4*>(hi)[e];
        if constexpr (C::kSplit) reinterpret_cast<uint4*>(wt_lo + off)[e] = reinterpret_cast<const uint4*>(lo)[e];
    }
}

// Plan store blocks (row-major FP32) -> B tiles (prepare time).
template <int MODE>
__global__ void tc_tile_kernel(const TileJob* __restrict__ jobs, const float* __restrict__ kstore,
                               const float* __restrict__ pstore, const int32_t* __restrict__ col_maps,
                               uint8_t* b_hi, uint8_t* b_lo) {
    using C = Cfg<MODE>;
    const TileJob jb = jobs[blockIdx.x];
    const float* src = (jb.src_store == A_KSTORE ? kstore : pstore) + jb.src_off;
    const int64_t per_chunk = int64_t(jb.n_pad) * C::kKc;
    for (int64_t e = threadIdx.x; e < per_chunk * jb.nchunks; e += blockDim.x) {
        const int ch = int(e / per_chunk);
        const int rem = int(e % per_chunk);
        const int n = rem / C::kKc, kk = rem % C::kKc;
        const int col = ch * C::kKc + kk;
        int sc = -1;
        if (jb.col_map_off >= 0) sc = col_maps[jb.col_map_off + col];
        else if (col < jb.k_split) sc = col;
        else if (col >= jb.k_split + jb.k_gap) sc = col - jb.k_gap;
        float x = 0.f;
        if (n < jb.m && sc >= 0 && sc < jb.k) x = src[int64_t(n) * jb.src_ld + sc];
        const int64_t at =
            jb.dst_off + int64_t(ch) * jb.n_pad * 128 + swz(uint32_t(n), uint32_t(kk * C::kEs), uint32_t(jb.n_pad));
        if constexpr (MODE == TC_TF32) {
            *reinterpret_cast<float*>(b_hi + at) = round_tf32(x);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            *reinterpret_cast<__nv_bfloat16*>(b_hi + at) = h;
            if constexpr (C::kSplit)
                *reinterpret_cast<__nv_bfloat16*>(b_lo + at) = __float2bfloat16_rn(x - __bfloat162float(h));
        }
    }
}

}  // namespace

// ------------------------------------------------------------------ host --
// One launch for every grouped GEMM of an evaluation.  Completion counters
// per (node, r-tile): w~ written (N2S), u~ written by S2S, u~ final (after
// the S2N push when there is one; with the S2N parent part pulled into the
// S2S task, as build_tc_plan does, that is the S2S task itself).  Each task waits for the counters of what
// it reads and bumps the counters of what it writes; tasks are ordered by
// the length of the dependent work that follows them (critical path first),
// which is a topological order.
// stage_mask selects the stages (bit 1 N2S, 2 S2S, 3 S2N, 4 leaves) whose
// tasks the launch runs; a dependency on a counter that no selected task
// bumps was satisfied by an earlier launch and is dropped.
static void build_fused(const Structure& st, TcPrec& T, TcFused& F, unsigned stage_mask) {
    const int64_t nn = st.n_nodes();
    constexpr int32_t E = 4;  // arrivals per task piece and r-tile: one per epilogue warp
    std::vector<int> pn2s(nn, 0), ps2s(nn, 0), ppush(nn, 0);
    for (const TcLaunch& l : T.launches)
        for (size_t k = 0; k < l.tasks.size(); ++k) {
            const int64_t h = l.task_node[k];
            if (l.stage == 1) ++pn2s[h];
            else if (l.stage == 2) ++ps2s[h];
            else if (l.stage == 3) ++ppush[h];
        }
    auto cWT = [&](int64_t h) { return int32_t(h); };
    auto cS2S = [&](int64_t h) { return int32_t(nn + h); };
    auto cUF = [&](int64_t h) { return int32_t(2 * nn + h); };
    auto final_pieces = [&](int64_t h) { return ppush[h] ? ppush[h] : ps2s[h]; };
    F.ncounters = int(3 * nn);
    // counters bumped inside this launch
    std::vector<char> internal(size_t(3 * nn), 0);
    for (const TcLaunch& l : T.launches) {
        if (!((stage_mask >> l.stage) & 1u)) continue;
        for (size_t k = 0; k < l.tasks.size(); ++k) {
            const int64_t h = l.task_node[k];
            if (l.stage == 1) internal[size_t(cWT(h))] = 1;
            else if (l.stage == 2) {
                internal[size_t(cS2S(h))] = 1;
                if (!ppush[h]) internal[size_t(cUF(h))] = 1;
            } else if (l.stage == 3) internal[size_t(cUF(h))] = 1;
        }
    }
    std::vector<int32_t> dep_off{0}, deps, sig;
    std::vector<int32_t> all_off{0}, all_deps;  // task and slab dependencies together (ordering only)
    std::vector<int64_t> work;
    std::vector<std::pair<int, int>> group;  // (stage, tree level) of every task
    std::vector<int64_t> node_of;
    F.piece = T.piece;
    F.wmax = T.gen && T.piece == 128 ? 4 : 2;  // the kernel variant's stage holds four r-tiles
    F.tasks.clear();
    F.slabs.clear();
    F.task_stage.clear();
    for (const TcLaunch& l : T.launches) {
        if (!((stage_mask >> l.stage) & 1u)) continue;
        for (size_t k = 0; k < l.tasks.size(); ++k) {
            TcTask t = l.tasks[k];
            const int32_t base = int32_t(F.slabs.size());
            // the counter that says a node's right-hand-side segment in a
            // buffer is complete: w~ after its N2S pieces, u~ when final
            auto operand_dep = [&](int32_t buf, int32_t node) -> std::pair<int32_t, int32_t> {
                if (node < 0 || buf == B_WT) return {-1, 0};
                if (buf == B_WTIL) return {cWT(node), E * pn2s[node]};
                return {cUF(node), E * final_pieces(node)};
            };
            std::vector<std::pair<int32_t, int32_t>> slab_deps;
            for (int si = t.slab0; si < t.slab1; ++si) {
                TcSlab sl = l.slabs[si];
                const auto d0 = operand_dep(sl.a_buf, sl.a_node0), d1 = operand_dep(sl.a_buf, sl.a_node1);
                if (d0.first >= 0 && internal[size_t(d0.first)]) {
                    sl.dep_c0 = d0.first;
                    sl.dep_n0 = d0.second;
                    slab_deps.push_back(d0);
                }
                if (d1.first >= 0 && internal[size_t(d1.first)]) {
                    sl.dep_c1 = d1.first;
                    sl.dep_n1 = d1.second;
                    slab_deps.push_back(d1);
                }
                F.slabs.push_back(sl);
            }
            t.slab1 = base + (t.slab1 - t.slab0);
            t.slab0 = base;
            const int64_t h = l.task_node[k];
            std::vector<std::pair<int32_t, int32_t>> d;  // (counter, arrivals needed)
            int32_t s0 = -1, s1 = -1;
            if (l.stage == 1) {
                if (!st.is_leaf(h)) {
                    d.emplace_back(cWT(2 * h + 1), E * pn2s[2 * h + 1]);
                    d.emplace_back(cWT(2 * h + 2), E * pn2s[2 * h + 2]);
                }
                s0 = cWT(h);
            } else if (l.stage == 2) {
                for (int64_t a : st.far[h]) d.emplace_back(cWT(a), E * pn2s[a]);
                s0 = cS2S(h);
                if (!ppush[h]) s1 = cUF(h);
            } else if (l.stage == 3) {
                const int64_t par = (h - 1) / 2;
                d.emplace_back(cS2S(h), E * ps2s[h]);
                d.emplace_back(cUF(par), E * final_pieces(par));
                s0 = cUF(h);
            } else if (ps2s[h] > 0) {  // leaf output reading u~ of the leaf
                d.emplace_back(cUF(h), E * final_pieces(h));
            }
            d.erase(std::remove_if(d.begin(), d.end(),
                                   [&](const std::pair<int32_t, int32_t>& x) { return !internal[size_t(x.first)]; }),
                    d.end());
            std::sort(d.begin(), d.end());
            d.erase(std::unique(d.begin(), d.end()), d.end());
            // the slabs' operand dependencies are waited for slab by slab in
            // the kernel (an S2S task's last slab, its parent's u~, only after
            // its far field); the rest (an S2N push waiting for its node's S2S
            // result) before the first copy
            for (auto& x : d) {
                if (std::find(slab_deps.begin(), slab_deps.end(), x) != slab_deps.end()) continue;
                deps.push_back(x.first);
                deps.push_back(x.second);
            }
            dep_off.push_back(int32_t(deps.size() / 2));
            for (auto& x : slab_deps) {  // all dependencies, for the orders computed below
                all_deps.push_back(x.first);
                all_deps.push_back(x.second);
            }
            for (auto& x : d) {
                if (std::find(slab_deps.begin(), slab_deps.end(), x) != slab_deps.end()) continue;
                all_deps.push_back(x.first);
                all_deps.push_back(x.second);
            }
            all_off.push_back(int32_t(all_deps.size() / 2));
            sig.push_back(s0);
            sig.push_back(s1);
            work.push_back(int64_t(t.nchunks) * t.n_pad);
            {
                int lev = 0;
                for (int64_t x = h + 1; x > 1; x >>= 1) ++lev;
                group.emplace_back(l.stage, lev);
                node_of.push_back(h);
                F.task_stage.push_back(int8_t(l.stage));
            }
            F.tasks.push_back(t);
        }
    }
    // priority: the longest chain of dependent work from a task to the end of
    // the evaluation (critical path first).  A producer's chain is longer
    // than any of its consumers', so the order stays topological.
    const size_t nt = F.tasks.size();
    std::vector<std::vector<int32_t>> consumers(size_t(F.ncounters));
    for (size_t t = 0; t < nt; ++t)
        for (int32_t d = all_off[t]; d < all_off[t + 1]; ++d)
            consumers[size_t(all_deps[2 * d])].push_back(int32_t(t));
    std::vector<int64_t> tail(nt, 0);
    for (size_t t = nt; t-- > 0;) {
        int64_t best = 0;
        for (int i = 0; i < 2; ++i) {
            const int32_t c = sig[2 * t + i];
            if (c < 0) continue;
            for (int32_t u : consumers[size_t(c)]) best = std::max(best, tail[size_t(u)]);
        }
        tail[t] = work[t] + 1024 + best;  // + per-tile overhead
    }
    F.order.resize(nt);
    for (size_t i = 0; i < nt; ++i) F.order[i] = int32_t(i);
    std::stable_sort(F.order.begin(), F.order.end(), [&](int32_t a, int32_t b) { return tail[a] > tail[b]; });

    // Locality order: a topological order (Kahn) that takes, among the ready
    // tasks, those of the (stage, tree level) group with the longest critical
    // path first and, inside a group, in heap order.  Neighbouring nodes share
    // most of their far (and near) lists, so consecutive tiles read the same
    // skeleton weights and the reads hit L2 instead of HBM.
    {
        std::vector<std::vector<int32_t>> producers(size_t(F.ncounters));
        for (size_t t = 0; t < nt; ++t)
            for (int i = 0; i < 2; ++i)
                if (sig[2 * t + i] >= 0) producers[size_t(sig[2 * t + i])].push_back(int32_t(t));
        std::map<std::pair<int, int>, int64_t> gmax;  // (stage, level) -> longest tail
        for (size_t t = 0; t < nt; ++t) {
            int64_t& g = gmax[group[t]];
            g = std::max(g, tail[t]);
        }
        std::vector<std::vector<int32_t>> succ(nt);
        std::vector<int32_t> indeg(nt, 0);
        for (size_t t = 0; t < nt; ++t) {
            std::vector<int32_t> pre;
            for (int32_t d = all_off[t]; d < all_off[t + 1]; ++d)
                for (int32_t u : producers[size_t(all_deps[2 * d])]) pre.push_back(u);
            std::sort(pre.begin(), pre.end());
            pre.erase(std::unique(pre.begin(), pre.end()), pre.end());
            for (int32_t u : pre) succ[size_t(u)].push_back(int32_t(t));
            indeg[t] = int32_t(pre.size());
        }
        // ready set ordered by (group's longest tail desc, stage, level, node, task)
        auto key = [&](int32_t t) {
            return std::make_tuple(-gmax[group[size_t(t)]], group[size_t(t)].first, group[size_t(t)].second,
                                   node_of[size_t(t)], t);
        };
        std::set<std::tuple<int64_t, int, int, int64_t, int32_t>> ready;
        for (size_t t = 0; t < nt; ++t)
            if (indeg[t] == 0) ready.insert(key(int32_t(t)));
        F.order_local.clear();
        while (!ready.empty()) {
            const int32_t t = std::get<4>(*ready.begin());
            ready.erase(ready.begin());
            F.order_local.push_back(t);
            for (int32_t u : succ[size_t(t)])
                if (--indeg[size_t(u)] == 0) ready.insert(key(u));
        }
        if (F.order_local.size() != nt) fail(GOFMM_ERR_ARG, "dependency cycle in the fused plan");

        // Schedule order: a list schedule simulated on the host.  A task runs
        // on one of W workers (the launch's CTAs over the two tiles a task
        // has at r = 512) for its work plus a per-tile overhead, and is ready
        // when every producer it waits for has finished.  The worker that
        // frees first takes, among the tasks ready by then, the first in the
        // locality order's priority (group with the longest critical path,
        // then heap order); if none is ready, the one ready first.  Taken only
        // after all its producers, so the order is topological; CTAs that
        // claim tiles in it find their operands ready more often than in a
        // priority order alone, and neighbouring tiles still share operands.
        const int workers = std::max(1, T.num_sms / 2);
        std::vector<int64_t> ready_at(nt, 0);
        std::vector<int32_t> left(indeg);
        using Ev = std::pair<int64_t, int32_t>;
        std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> pending;  // (ready time, task)
        std::set<std::tuple<int64_t, int, int, int64_t, int32_t>> avail;      // locality priority
        std::priority_queue<int64_t, std::vector<int64_t>, std::greater<int64_t>> freeat;
        for (int w = 0; w < workers; ++w) freeat.push(0);
        for (size_t t = 0; t < nt; ++t)
            if (left[t] == 0) pending.push({0, int32_t(t)});
        F.order_sched.clear();
        while (F.order_sched.size() < nt) {
            int64_t now = freeat.top();
            freeat.pop();
            if (avail.empty() && !pending.empty() && pending.top().first > now) now = pending.top().first;
            while (!pending.empty() && pending.top().first <= now) {
                avail.insert(key(pending.top().second));
                pending.pop();
            }
            if (avail.empty()) fail(GOFMM_ERR_ARG, "dependency cycle in the fused plan");
            const int32_t t = std::get<4>(*avail.begin());
            avail.erase(avail.begin());
            const int64_t done = now + work[size_t(t)] + 1024;
            freeat.push(done);
            F.order_sched.push_back(t);
            for (int32_t u : succ[size_t(t)]) {
                ready_at[size_t(u)] = std::max(ready_at[size_t(u)], done);
                if (--left[size_t(u)] == 0) pending.push({ready_at[size_t(u)], u});
            }
        }
    }
    // Level order: the upward pass (as in the locality order), then the S2S
    // tasks level by level from the top (heap order inside a level), with
    // S2N pushes into level l, where a plan has them, placed after the S2S
    // tasks of level l + 1; then the leaves.  With the parent part pulled
    // into each S2S task (build_tc_plan) a node's task is claimed a whole
    // level after its parent's, so its wait before the last slab is short.
    // Topological (checked below).
    {
        int L = 0;
        for (size_t t = 0; t < nt; ++t) L = std::max(L, group[t].second);
        std::vector<std::vector<int32_t>> s2s(size_t(L) + 1), push(size_t(L) + 1);
        std::vector<int32_t> up, leaves;
        for (int32_t t : F.order_local) {
            const int stg = group[size_t(t)].first, lev = group[size_t(t)].second;
            if (stg == 1) up.push_back(t);
            else if (stg == 2) s2s[size_t(lev)].push_back(t);
            else if (stg == 3) push[size_t(lev)].push_back(t);
            else leaves.push_back(t);
        }
        auto heap = [&](std::vector<int32_t>& v) {
            std::stable_sort(v.begin(), v.end(),
                             [&](int32_t a, int32_t b) { return node_of[size_t(a)] < node_of[size_t(b)]; });
        };
        F.order_levels = up;
        for (int l = 0; l <= L; ++l) {
            heap(s2s[size_t(l)]);
            F.order_levels.insert(F.order_levels.end(), s2s[size_t(l)].begin(), s2s[size_t(l)].end());
            if (l >= 1) {
                heap(push[size_t(l - 1)]);
                F.order_levels.insert(F.order_levels.end(), push[size_t(l - 1)].begin(), push[size_t(l - 1)].end());
            }
        }
        heap(push[size_t(L)]);
        F.order_levels.insert(F.order_levels.end(), push[size_t(L)].begin(), push[size_t(L)].end());
        F.order_levels.insert(F.order_levels.end(), leaves.begin(), leaves.end());
        if (F.order_levels.size() != nt) fail(GOFMM_ERR_ARG, "level order does not cover the fused plan");
        std::vector<int64_t> pos(nt);
        for (size_t i = 0; i < nt; ++i) pos[size_t(F.order_levels[i])] = int64_t(i);
        std::vector<std::vector<int32_t>> prod(size_t(F.ncounters));
        for (size_t t = 0; t < nt; ++t)
            for (int i = 0; i < 2; ++i)
                if (sig[2 * t + i] >= 0) prod[size_t(sig[2 * t + i])].push_back(int32_t(t));
        for (size_t t = 0; t < nt; ++t)
            for (int32_t d = all_off[t]; d < all_off[t + 1]; ++d)
                for (int32_t u : prod[size_t(all_deps[2 * d])])
                    if (pos[size_t(u)] > pos[t]) fail(GOFMM_ERR_ARG, "level order is not topological");
    }
    F.d_tasks = dupload(F.tasks);
    F.d_slabs = dupload(F.slabs);
    F.d_dep_off = dupload(dep_off);
    F.dep_off_host = dep_off;
    F.deps_host = deps;
    F.d_deps = dupload(deps.empty() ? std::vector<int32_t>{0, 0} : deps);
    F.d_sig = dupload(sig);
}

// Ready-queue form of the fused launch for n_rtiles r-tiles: the upward
// pass and S2S tiles in the locality order (claimed in list order), then the
// push (where a plan has them) and leaf tiles, which enter the launch's
// queue once complete: for
// each of them the (counter, r-tile) pairs it waits for (its task's
// dependencies and its slabs' operand counters over its r-tiles), inverted
// into per-pair consumer lists; those with none start in the queue.
static TcFused::Ready& ready_tiles(TcFused& F, int n_rtiles) {
    auto it = F.ready.find(n_rtiles);
    if (it != F.ready.end()) return it->second;
    std::vector<TcTile> tiles, queued;
    std::vector<int32_t> qtask;
    for (int32_t k : F.order_local) {
        const bool q = F.task_stage[size_t(k)] >= 3;
        const size_t before = q ? queued.size() : tiles.size();
        task_tiles(q ? queued : tiles, 0, k, F.tasks[size_t(k)], n_rtiles, F.wmax);
        if (q)
            for (size_t i = before; i < queued.size(); ++i) qtask.push_back(k);
    }
    TcFused::Ready R;
    R.n_static = int(tiles.size());
    R.n = int(queued.size());
    const size_t npairs = size_t(F.ncounters) * size_t(n_rtiles);
    std::vector<int32_t> req(size_t(F.ncounters), 0), pending(size_t(R.n), 0);
    std::vector<std::vector<int32_t>> cons(npairs);
    auto need = [&](int32_t c, int32_t e) {
        if (req[size_t(c)] != 0 && req[size_t(c)] != e) fail(GOFMM_ERR_ARG, "inconsistent counter target in the fused plan");
        req[size_t(c)] = e;
    };
    for (int i = 0; i < R.n; ++i) {
        const TcTile& t = queued[size_t(i)];
        const int32_t k = qtask[size_t(i)];
        std::vector<std::pair<int32_t, int32_t>> d;  // (counter, arrivals)
        for (int32_t x = F.dep_off_host[size_t(k)]; x < F.dep_off_host[size_t(k) + 1]; ++x)
            d.emplace_back(F.deps_host[size_t(2 * x)], F.deps_host[size_t(2 * x + 1)]);
        const TcTask& tk = F.tasks[size_t(k)];
        for (int si = tk.slab0; si < tk.slab1; ++si) {
            const TcSlab& sl = F.slabs[size_t(si)];
            if (sl.dep_c0 >= 0) d.emplace_back(sl.dep_c0, sl.dep_n0);
            if (sl.dep_c1 >= 0) d.emplace_back(sl.dep_c1, sl.dep_n1);
        }
        std::sort(d.begin(), d.end());
        d.erase(std::unique(d.begin(), d.end()), d.end());
        for (const auto& x : d) {
            need(x.first, x.second);
            for (int w = 0; w < tile_width_host(t); ++w) {
                cons[size_t(x.first) * size_t(n_rtiles) + size_t(t.rt + w)].push_back(i);
                ++pending[size_t(i)];
            }
        }
    }
    std::vector<int32_t> off(npairs + 1, 0), flat;
    for (size_t pidx = 0; pidx < npairs; ++pidx) {
        off[pidx + 1] = off[pidx] + int32_t(cons[pidx].size());
        flat.insert(flat.end(), cons[pidx].begin(), cons[pidx].end());
    }
    std::vector<int> q0(size_t(2 + R.n), -1);
    int ready0 = 0;
    for (int i = 0; i < R.n; ++i)
        if (pending[size_t(i)] == 0) q0[size_t(2 + ready0++)] = R.n_static + i;
    q0[0] = ready0;  // tail
    q0[1] = 0;       // head
    tiles.insert(tiles.end(), queued.begin(), queued.end());
    R.tiles = dupload(tiles);
    R.queue0 = dupload(q0);
    R.queue = dalloc<int>(q0.size());
    R.pending0 = dupload(pending.empty() ? std::vector<int32_t>{0} : pending);
    R.pending = dalloc<int>(std::max<size_t>(pending.size(), 1));
    R.cons_off = dupload(off);
    R.cons = dupload(flat.empty() ? std::vector<int32_t>{0} : flat);
    R.req = dupload(req);
    return F.ready.emplace(n_rtiles, R).first->second;
}

// Tile list of the fused launch: tasks in the given order (GOFMM_ORDER_*),
// the r-tiles of a task adjacent.
static std::pair<TcTile*, int> fused_tiles(TcFused& F, int n_rtiles, int order) {
    const int key = n_rtiles * 8 + order;  // GOFMM_ORDER_* < 8
    auto it = F.tiles.find(key);
    if (it != F.tiles.end()) return it->second;
    std::vector<TcTile> t;
    for (int32_t k : fused_order(F, order))
        task_tiles(t, 0, k, F.tasks[size_t(k)], n_rtiles, F.wmax);
    auto v = std::make_pair(dupload(t), int(t.size()));
    F.tiles[key] = v;
    return v;
}

static void build_tc_plan(const Structure& st, DeviceState& D, TcPrec& T, std::vector<TileJob>& jobs,
                          std::vector<int32_t>& col_maps) {
    const int64_t nn = st.n_nodes(), nl = st.n_leaves();
    const int kc = T.kc;
    const int64_t P = T.piece;
    if (P != 128 && P != 256) fail(GOFMM_ERR_ARG, "task piece height must be 128 or 256");
    auto padk = [&](int64_t x) { return (x + kc - 1) / kc * kc; };
    std::vector<int64_t> leaf_chunk(nl), node_chunk(nn, -1);
    std::map<int64_t, int64_t> leaf_at_pos, node_at_skel;
    int64_t c = 0;
    std::vector<int64_t> chunk_pos;
    std::vector<int32_t> chunk_valid;
    for (int64_t b = 0; b < nl; ++b) {
        const int64_t h = st.leaf_node(b);
        leaf_chunk[b] = c;
        leaf_at_pos[st.node_off[h]] = b;
        for (int64_t i = 0; i < st.node_size[h]; i += kc) {
            chunk_pos.push_back(st.node_off[h] + i);
            chunk_valid.push_back(int32_t(std::min<int64_t>(kc, st.node_size[h] - i)));
        }
        c += padk(st.node_size[h]) / kc;
    }
    T.wt_chunks = c;
    c = 0;
    for (int64_t h = 1; h < nn; ++h) {
        node_chunk[h] = c;
        node_at_skel[D.skel_off[h]] = h;
        c += padk(int64_t(st.skel[h].size())) / kc;
    }
    T.sk_chunks = std::max<int64_t>(c, 1);
    T.d_chunk_pos = dupload(chunk_pos);
    T.d_chunk_valid = dupload(chunk_valid);

    int64_t bbytes = 0;
    T.launches.clear();
    // one task of the plan with the given slabs, as task pieces of at most P
    // rows; a slab may carry a column map of its block (SlabRef::cmap, with
    // SlabRef::kpad columns in chunks of kc)
    struct SlabRef {
        const Slab* s;
        int64_t cmap = -1, kpad = -1;
    };
    auto emit = [&](TcLaunch& tl, const Task& t, const std::vector<SlabRef>& slabs, bool acc) {
        int64_t out_base;
        const int okind = task_out(t.flags);
        if (okind == OUT_U) out_base = t.out_row;
        else out_base = node_chunk.at(node_at_skel.at(t.out_row));
        for (int64_t q = 0; q * P < std::max<int64_t>(t.m, 1); ++q) {
            const int32_t mq = int32_t(std::min<int64_t>(P, t.m - q * P));
            TcTask tt{};
            tt.out_pos = okind == OUT_U ? out_base + q * P : out_base + q * P / kc;
            tt.m = mq;
            tt.n_pad = std::max(16, (mq + 15) / 16 * 16);
            tt.slab0 = int32_t(tl.slabs.size());
            tt.out_kind = okind;
            tt.accumulate = acc ? 1 : 0;
            tt.out_cols = okind == OUT_U ? tt.n_pad : int32_t(std::min<int64_t>(P, padk(t.m) - q * P));
            for (const SlabRef& ref : slabs) {
                const Slab& s = *ref.s;
                TcSlab ts{};
                ts.a_buf = s.b_src;
                ts.a_node0 = ts.a_node1 = -1;
                ts.dep_c0 = ts.dep_c1 = -1;
                if (s.b_src != B_WT) {
                    const int64_t a = node_at_skel.at(s.b_row);
                    ts.a_node0 = int32_t(a);
                    if (s.k != int64_t(st.skel[a].size())) ts.a_node1 = int32_t(a + 1);  // [w~_l; w~_r]
                }
                if (s.a_src == A_GEN) {
                    // block entries generated in the kernel from the row
                    // list (this piece's rows) and the column list
                    const int64_t a = s.b_src == B_WT ? leaf_at_pos.at(s.b_row) : node_at_skel.at(s.b_row);
                    ts.a_chunk0 = int32_t(s.b_src == B_WT ? leaf_chunk[a] : node_chunk[a]);
                    ts.nchunks = int32_t(padk(s.k) / kc);
                    ts.gen = 1;
                    ts.b_off = s.a_off + q * P;
                    ts.gen_cols = s.a_col;
                    ts.k = s.k;
                    T.gen = true;
                    tt.nchunks += ts.nchunks;
                    tl.slabs.push_back(ts);
                    continue;
                }
                int64_t ksplit = s.k, kgap = 0, kpad;
                if (s.b_src == B_WT) {
                    const int64_t a = leaf_at_pos.at(s.b_row);
                    ts.a_chunk0 = int32_t(leaf_chunk[a]);
                    kpad = ref.kpad >= 0 ? ref.kpad : padk(s.k);
                } else {
                    const int64_t a = node_at_skel.at(s.b_row);
                    const int64_t sa = int64_t(st.skel[a].size());
                    ts.a_chunk0 = int32_t(node_chunk[a]);
                    if (s.k == sa) {
                        kpad = padk(sa);
                    } else {  // [w~_l; w~_r]: two adjacent sibling segments
                        const int64_t sb = int64_t(st.skel[a + 1].size());
                        if (s.k != sa + sb || node_chunk[a + 1] != node_chunk[a] + padk(sa) / kc)
                            fail(GOFMM_ERR_ARG, "unexpected slab layout in the tensor-core plan");
                        ksplit = sa;
                        kgap = padk(sa) - sa;
                        kpad = padk(sa) + padk(sb);
                    }
                }
                ts.nchunks = int32_t(kpad / kc);
                ts.b_off = bbytes;
                TileJob jb{};
                jb.src_off = s.a_off + q * P * int64_t(s.lda);
                jb.dst_off = bbytes;
                jb.col_map_off = ref.cmap;
                jb.src_ld = s.lda;
                jb.m = mq;
                jb.k = s.k;
                jb.n_pad = tt.n_pad;
                jb.nchunks = ts.nchunks;
                jb.k_split = int32_t(ksplit);
                jb.k_gap = int32_t(kgap);
                jb.src_store = s.a_src;
                jobs.push_back(jb);
                bbytes += int64_t(ts.nchunks) * tt.n_pad * 128;
                tt.nchunks += ts.nchunks;
                tl.slabs.push_back(ts);
            }
            tt.slab1 = int32_t(tl.slabs.size());
            tl.tasks.push_back(tt);
            tl.task_node.push_back(okind == OUT_U ? st.leaf_node(leaf_at_pos.at(t.out_row))
                                                  : node_at_skel.at(t.out_row));
        }
    };
    // Full-rank subtrees.  A node whose rank is its column count (ncols =
    // s) has P = Pi^T, a permutation, and if its children are full rank too,
    // w~ of the node is W itself: row k of w~ is the row of W at tree
    // position tpos[h][k].  A slab that reads w~ of such nodes then reads W
    // (tree order) instead, its block's columns permuted to match (a column
    // map applied when the block tiles are made; generated blocks take the
    // tree-order column list): the same products, with no N2S task to wait
    // for.  N2S tasks whose output nobody reads any more are dropped.
    std::vector<std::vector<int64_t>> tpos(static_cast<size_t>(nn));
    for (int64_t h = nn - 1; h >= 1; --h) {
        const int64_t sh = int64_t(st.skel[h].size()), nc = st.ncols(h);
        if (sh != nc || int64_t(st.P[h].size()) != sh * nc) continue;
        if (!st.is_leaf(h) && (tpos[2 * h + 1].empty() || tpos[2 * h + 2].empty())) continue;
        std::vector<int64_t> v(size_t(sh), -1);
        bool perm_ok = true;
        for (int64_t k = 0; k < sh && perm_ok; ++k) {
            int64_t c1 = -1;
            for (int64_t c = 0; c < nc && perm_ok; ++c) {
                const double x = st.P[h][size_t(k * nc + c)];
                if (x == 1.0 && c1 < 0) c1 = c;
                else if (x != 0.0) perm_ok = false;
            }
            if (c1 < 0) { perm_ok = false; break; }
            if (st.is_leaf(h)) v[size_t(k)] = st.node_off[h] + c1;
            else {
                const int64_t sl = int64_t(st.skel[2 * h + 1].size());
                v[size_t(k)] = c1 < sl ? tpos[2 * h + 1][size_t(c1)] : tpos[2 * h + 2][size_t(c1 - sl)];
            }
        }
        if (perm_ok) tpos[h] = std::move(v);
    }
    std::vector<std::vector<Slab>> dslabs(D.launches.size());
    std::vector<std::vector<int64_t>> dcmap(D.launches.size()), dkpad(D.launches.size());
    for (size_t li = 0; li < D.launches.size(); ++li) {
        const Launch& l = D.launches[li];
        dslabs[li] = l.slabs;
        dcmap[li].assign(l.slabs.size(), -1);
        dkpad[li].assign(l.slabs.size(), -1);
        for (size_t si = 0; si < l.slabs.size(); ++si) {
            Slab& sl = dslabs[li][si];
            if (sl.b_src != B_WTIL) continue;
            const int64_t a = node_at_skel.at(sl.b_row);
            const bool two = sl.k != int64_t(st.skel[a].size());
            if (tpos[a].empty() || (two && tpos[a + 1].empty())) continue;
            // tree positions of the slab's right-hand-side rows: the leaves
            // of the node (or of both siblings), consecutive
            const int64_t t0 = st.node_off[a];
            const int64_t b0 = leaf_at_pos.at(t0);
            std::vector<int64_t> inv(size_t(sl.k), -1);  // tree position - t0 -> slab column
            const int64_t sa = int64_t(st.skel[a].size());
            for (int64_t c = 0; c < sl.k; ++c) {
                const int64_t tp = c < sa ? tpos[a][size_t(c)] : tpos[a + 1][size_t(c - sa)];
                if (tp < t0 || tp >= t0 + sl.k || inv[size_t(tp - t0)] >= 0)
                    fail(GOFMM_ERR_ARG, "full-rank subtree rows out of place in the tensor-core plan");
                inv[size_t(tp - t0)] = int32_t(c);
            }
            // the chunk layout of W in tree order: each leaf padded to whole chunks
            std::vector<int32_t> map;
            bool gapless = true;
            for (int64_t b = b0, done = 0; done < sl.k; ++b) {
                const int64_t h = st.leaf_node(b), ns = st.node_size[h];
                if (done + ns < sl.k && ns % kc != 0) gapless = false;
                for (int64_t i = 0; i < padk(ns); ++i)
                    map.push_back(i < ns ? int32_t(inv[size_t(done + i)]) : -1);
                done += ns;
            }
            if (sl.a_src == A_GEN) {
                // generated blocks: the column list in tree order (no map),
                // when the leaves leave no padding inside the range
                if (!gapless) continue;
                sl.a_col = t0;
            } else {
                dcmap[li][si] = int64_t(col_maps.size());
                dkpad[li][si] = int64_t(map.size());
                col_maps.insert(col_maps.end(), map.begin(), map.end());
            }
            sl.b_src = B_WT;
            sl.b_row = t0;
        }
    }
    std::vector<char> wtil_read(static_cast<size_t>(nn), 0);
    for (size_t li = 0; li < D.launches.size(); ++li)
        for (const Slab& sl : dslabs[li])
            if (sl.b_src == B_WTIL) {
                const int64_t a = node_at_skel.at(sl.b_row);
                wtil_read[size_t(a)] = 1;
                if (sl.k != int64_t(st.skel[a].size())) wtil_read[size_t(a + 1)] = 1;
            }
    // The downward pass pulls instead of pushing: a node's S2S task takes
    // the S2N slab of its parent's push into it, (P^T_{p~[l~r~]})[rows of the
    // node] u~_p, as its last slab, so u~ of the node is written once, final
    // (far field + parent part, one accumulation).  Every task of a level
    // then reads its parent's final u~: the per-stage launches run the S2S
    // tasks level by level from the top, and a dependency-driven launch
    // waits for the parent only before that last slab, after the node's far
    // field.  The separate in-place S2N launches go away.
    std::map<int64_t, const Slab*> pull;  // node -> its parent's push slab into it
    for (const Launch& l : D.launches)
        if (l.stage == 3)
            for (const Task& t : l.tasks) {
                if (t.slab1 - t.slab0 != 1) fail(GOFMM_ERR_ARG, "unexpected S2N task in the tensor-core plan");
                pull[node_at_skel.at(t.out_row)] = &l.slabs[size_t(t.slab0)];
            }
    for (size_t li = 0; li < D.launches.size(); ++li) {
        const Launch& l = D.launches[li];
        if (l.stage == 3) continue;
        auto slabs_of = [&](const Task& t) {
            std::vector<SlabRef> v;
            for (int si = t.slab0; si < t.slab1; ++si)
                v.push_back(SlabRef{&dslabs[li][size_t(si)], dcmap[li][size_t(si)], dkpad[li][size_t(si)]});
            return v;
        };
        if (l.stage != 2) {
            TcLaunch tl;
            tl.stage = l.stage;
            for (const Task& t : l.tasks) {
                // an N2S task whose w~ no slab reads (its readers take W)
                if (l.stage == 1 && !wtil_read[size_t(node_at_skel.at(t.out_row))]) continue;
                emit(tl, t, slabs_of(t), task_accumulate(t.flags));
            }
            tl.piece = T.piece;
            T.launches.push_back(std::move(tl));
            continue;
        }
        // S2S: one launch per tree level, top-down (the order inside a level kept)
        std::map<int, TcLaunch> lv;
        for (const Task& t : l.tasks) {
            const int64_t h = node_at_skel.at(t.out_row);
            int lev = 0;
            for (int64_t x = h + 1; x > 1; x >>= 1) ++lev;
            auto v = slabs_of(t);
            const auto it = pull.find(h);
            if (it != pull.end()) v.push_back(SlabRef{it->second});
            TcLaunch& tl = lv[lev];
            tl.stage = 2;
            emit(tl, t, v, task_accumulate(t.flags));
            pull.erase(h);
        }
        for (auto& e : lv) {
            e.second.piece = T.piece;
            T.launches.push_back(std::move(e.second));
        }
    }
    if (!pull.empty()) fail(GOFMM_ERR_ARG, "an S2N push into a node without an S2S task");
    T.b_bytes = bbytes;
    for (TcLaunch& l : T.launches) l.wmax = T.gen && P == 128 ? 4 : 2;  // as the fused plans below
    // every range a kernel will touch, checked on the host before upload
    auto check = [](bool ok, const char* what) {
        if (!ok) fail(GOFMM_ERR_ARG, std::string("tensor-core plan out of range: ") + what);
    };
    const int64_t chunks[3] = {T.wt_chunks, T.sk_chunks, T.sk_chunks};
    for (const TcLaunch& l : T.launches)
        for (const TcTask& t : l.tasks) {
            check(t.m >= 1 && t.m <= P && t.n_pad % 16 == 0 && t.n_pad >= t.m && t.n_pad <= P, "task shape");
            check(t.slab0 >= 0 && t.slab0 <= t.slab1 && t.slab1 <= int32_t(l.slabs.size()), "task slabs");
            if (t.out_kind == OUT_U)
                check(t.out_pos >= 0 && t.out_pos + t.m <= st.n, "output rows");
            else
                check(t.out_pos >= 0 && t.out_cols % 32 == 0 && t.out_cols >= t.n_pad &&
                          t.out_pos + t.out_cols / kc <= T.sk_chunks, "output chunks");
            int64_t total = 0;
            for (int si = t.slab0; si < t.slab1; ++si) {
                const TcSlab& sl = l.slabs[si];
                check(sl.a_buf >= 0 && sl.a_buf < 3, "operand buffer");
                check(sl.a_chunk0 >= 0 && sl.a_chunk0 + sl.nchunks <= chunks[sl.a_buf], "operand chunks");
                if (sl.gen) {
                    const int64_t n_idx = st.n + D.S_tot;
                    check(sl.b_off >= 0 && sl.b_off + t.m <= n_idx && sl.gen_cols >= 0 && sl.gen_cols + sl.k <= n_idx &&
                              sl.k >= 1 && int64_t(sl.nchunks) * kc >= sl.k && int64_t(sl.nchunks - 1) * kc < sl.k,
                          "generated slab");
                } else {
                    check(sl.b_off % 16 == 0 && sl.b_off + int64_t(sl.nchunks) * t.n_pad * 128 <= T.b_bytes,
                          "B tiles");
                }
                total += sl.nchunks;
            }
            check(total == t.nchunks, "chunk count");
        }
    for (const TileJob& j : jobs) {
        const int64_t lim = j.src_store == A_KSTORE ? D.kstore_elems : D.pstore_elems;
        check(j.m >= 1 && j.k >= 1 && j.k <= j.src_ld, "tile job shape");
        check(j.src_off >= 0 && j.src_off + int64_t(j.m - 1) * j.src_ld + j.k <= lim, "tile job source");
        check(j.dst_off + int64_t(j.nchunks) * j.n_pad * 128 <= T.b_bytes, "tile job destination");
        check(int64_t(j.nchunks) * T.kc >= int64_t(j.k_split) + j.k_gap + (j.k - j.k_split), "tile job columns");
    }
    for (TcLaunch& l : T.launches) {
        l.d_tasks = dupload(l.tasks);
        l.d_slabs = dupload(l.slabs);
    }
    build_fused(st, T, T.fused, 0x1Eu);               // every stage
    build_fused(st, T, T.fused_up, 1u << 1);          // the upward pass
    build_fused(st, T, T.fused_down, (1u << 3) | (1u << 4));  // the downward pass and the leaves
}

template <int MODE>
static void set_smem_attr() {
    CUDA_OK(cudaFuncSetAttribute(tc_gemm_kernel<MODE, 256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 gemm_smem<MODE, 256, false>()));
    CUDA_OK(cudaFuncSetAttribute(tc_gemm_kernel<MODE, 128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 gemm_smem<MODE, 128, false>()));
    CUDA_OK(cudaFuncSetAttribute(tc_gemm_kernel<MODE, 256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 gemm_smem<MODE, 256, true>()));
    CUDA_OK(cudaFuncSetAttribute(tc_gemm_kernel<MODE, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 gemm_smem<MODE, 128, true>()));
    CUDA_OK(cudaFuncSetAttribute(tc_gemm_pair_kernel<MODE, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 Cfg2<MODE, 256>::kSmem));
    CUDA_OK(cudaFuncSetAttribute(tc_gemm_pair_kernel<MODE, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 Cfg2<MODE, 128>::kSmem));
}

// Tile list of one launch alone, the r-tiles of a task adjacent so they
// share the task's B tiles through L2.  CRITICAL: tasks in plan order
// (heaviest first, for the tail of the launch); LOCAL: tasks in heap order
// (tree levels top down, nodes left to right), so that consecutive tasks
// share most of their far or near lists and re-read operands from L2.
// With pair = true the list holds pairs of r-tiles (rt = pair index) for the
// SM-pair kernel.
std::pair<TcTile*, int> launch_tiles(TcLaunch& l, int n_rtiles, int order, bool pair, int wmax) {
    if (pair) n_rtiles = (n_rtiles + 1) / 2;
    const int key = (n_rtiles * 4 + (order != GOFMM_ORDER_CRITICAL ? 1 : 0) + (pair ? 2 : 0)) * 8 + wmax;
    auto it = l.tiles.find(key);
    if (it != l.tiles.end()) return it->second;
    std::vector<int32_t> tasks(l.tasks.size());
    for (size_t k = 0; k < tasks.size(); ++k) tasks[k] = int32_t(k);
    if (order != GOFMM_ORDER_CRITICAL)  // heap order
        std::stable_sort(tasks.begin(), tasks.end(),
                         [&](int32_t a, int32_t b) { return l.task_node[size_t(a)] < l.task_node[size_t(b)]; });
    std::vector<TcTile> t;
    for (int32_t k : tasks) {
        if (pair)  // a tile is one r-tile pair of the SM-pair kernel
            for (int rt = 0; rt < n_rtiles; ++rt) t.push_back(TcTile{0, k, rt, 0});
        else
            task_tiles(t, 0, k, l.tasks[size_t(k)], n_rtiles, wmax);
    }
    auto v = std::make_pair(dupload(t), int(t.size()));
    l.tiles[key] = v;
    return v;
}

static void occupancy_pairs(int num_sms);

TcPrec& tc_plan(Handle& H, DeviceState& D, int precision) {
    if (!D.tc) D.tc = new TcState();
    const int mode = mode_of(precision);
    TcPrec*& T = D.tc->prec[mode];
    if (!T) {
        auto t = std::make_unique<TcPrec>();
        t->mode = mode;
        t->kc = mode == TC_TF32 ? 32 : 64;
        t->es = mode == TC_TF32 ? 4 : 2;
        t->split = mode == TC_BF16X3;
        t->piece = H.tc_piece[mode];
        int dev = 0;
        CUDA_OK(cudaGetDevice(&dev));
        CUDA_OK(cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, dev));  // the plan's orders use it
        std::vector<TileJob> jobs;
        std::vector<int32_t> col_maps;
        build_tc_plan(H.st, D, *t, jobs, col_maps);
        if (t->gen) {
            // point table in index-list order for the generator warps: the
            // coordinates in FP32, then the squared norm of those FP32
            // coordinates (summed in FP64, rounded once), zero padding to a
            // multiple of four floats
            if (H.K.dim + 1 > kGenMaxDpad)
                fail(GOFMM_ERR_UNSUPPORTED, "in-kernel generation on the tensor cores supports at most 15 coordinates");
            const int dp = (H.K.dim + 1 + 3) / 4 * 4;
            std::vector<float> tab(D.idx.size() * size_t(dp), 0.f);
            for (size_t q = 0; q < D.idx.size(); ++q) {
                double nrm = 0.0;
                for (int d = 0; d < H.K.dim; ++d) {
                    const float x = float(H.K.pts[size_t(D.idx[q]) * size_t(H.K.dim) + size_t(d)]);
                    tab[q * size_t(dp) + size_t(d)] = x;
                    nrm += double(x) * double(x);
                }
                tab[q * size_t(dp) + size_t(H.K.dim)] = float(nrm);
            }
            t->gen_pts = dupload(tab);
            t->gen_dim = H.K.dim;
            t->gen_dpad = dp;
            t->gen_kind = H.K.kind;
            t->gen_inv = float(H.K.kind == GOFMM_GEN_GAUSSIAN ? 1.0 / (2.0 * H.K.h * H.K.h) : 1.0 / (H.K.h * H.K.h));
            t->gen_shift = float(H.K.shift);
        }
        t->b_hi = dalloc<uint8_t>(size_t(std::max<int64_t>(t->b_bytes, 16)));
        if (t->split) t->b_lo = dalloc<uint8_t>(size_t(std::max<int64_t>(t->b_bytes, 16)));
        if (!jobs.empty()) {
            TileJob* dj = dupload(jobs);
            int32_t* dm = dupload(col_maps.empty() ? std::vector<int32_t>{-1} : col_maps);
            const float* ks = static_cast<const float*>(D.fam[1].kstore);
            const float* ps = static_cast<const float*>(D.fam[1].pstore);
            const unsigned nj = unsigned(jobs.size());
            if (mode == TC_TF32) tc_tile_kernel<TC_TF32><<<nj, 256>>>(dj, ks, ps, dm, t->b_hi, t->b_lo);
            else if (mode == TC_BF16) tc_tile_kernel<TC_BF16><<<nj, 256>>>(dj, ks, ps, dm, t->b_hi, t->b_lo);
            else tc_tile_kernel<TC_BF16X3><<<nj, 256>>>(dj, ks, ps, dm, t->b_hi, t->b_lo);
            CUDA_OK(cudaGetLastError());
            CUDA_OK(cudaDeviceSynchronize());
            dfree(dj);
            dfree(dm);
        }
        t->d_err = dalloc<int>(1);
        CUDA_OK(cudaMemset(t->d_err, 0, sizeof(int)));
        t->d_claims = dalloc<int>(kClaimSlots);
        CUDA_OK(cudaMallocHost(&t->h_err, sizeof(int)));
        *t->h_err = 0;
        set_smem_attr<TC_TF32>();
        set_smem_attr<TC_BF16>();
        set_smem_attr<TC_BF16X3>();
        occupancy_pairs(t->num_sms);  // before any stream capture
        T = t.release();
    }
    return *T;
}

void tc_prepare(Handle& H, DeviceState& D, int64_t r_max, int precision) {
    TcPrec* T = &tc_plan(H, D, precision);
    const int64_t r_pad = (r_max + 127) / 128 * 128;
    // every r-tile count up to the prepared one (the serving engine mixes r)
    for (TcLaunch& l : T->launches)
        for (int nrt = 1; nrt <= int(r_pad / 128); ++nrt)
            launch_tiles(l, nrt, H.tc_order[T->mode], H.tc_schedule[T->mode] == GOFMM_SCHED_PAIR,
                         H.tc_schedule[T->mode] == GOFMM_SCHED_PAIR ? 2 : l.wmax);
    for (TcFused* F : {&T->fused, &T->fused_up, &T->fused_down}) {
        if (F->counters_nrt < int(r_pad / 128)) {
            dfree(F->d_counters);
            F->d_counters = dalloc<int>(size_t(F->ncounters) * size_t(r_pad / 128) + 1);  // + tile counter
            F->counters_nrt = int(r_pad / 128);
        }
        for (int nrt = 1; nrt <= int(r_pad / 128); ++nrt) {
            fused_tiles(*F, nrt, H.tc_order[T->mode]);
            if (H.tc_order[T->mode] == GOFMM_ORDER_READY && !F->tasks.empty()) ready_tiles(*F, nrt);
        }
    }
    if (T->r_cap < r_pad) {
        for (int i = 0; i < 3; ++i) {
            dfree(T->rt_hi[i]);
            dfree(T->rt_lo[i]);
            T->rt_hi[i] = T->rt_lo[i] = nullptr;
        }
        T->r_cap = 0;
        const int64_t chunks[3] = {T->wt_chunks, T->sk_chunks, T->sk_chunks};
        for (int i = 0; i < 3; ++i) {
            const size_t bytes = size_t(r_pad / 128) * size_t(chunks[i]) * kTileBytes;
            T->rt_hi[i] = dalloc<uint8_t>(bytes);
            CUDA_OK(cudaMemset(T->rt_hi[i], 0, bytes));
            if (T->split) {
                T->rt_lo[i] = dalloc<uint8_t>(bytes);
                CUDA_OK(cudaMemset(T->rt_lo[i], 0, bytes));
            }
        }
        T->r_cap = r_pad;
    }
}

bool tc_ready(const DeviceState& D, int64_t r, int precision) {
    if (!D.tc) return false;
    const TcPrec* T = D.tc->prec[mode_of(precision)];
    return T && T->r_cap >= r;
}

// Segment of one launch of one compressed matrix evaluated into the given
// RT buffers and output.
TcSeg make_seg(const TcPrec& T, const TcLaunch& l, uint8_t* const* rt_hi, uint8_t* const* rt_lo, float* U,
                      int64_t ldu, const int64_t* perm, int r) {
    TcSeg g{};
    g.tasks = l.d_tasks;
    g.slabs = l.d_slabs;
    g.b_hi = T.b_hi;
    g.b_lo = T.b_lo;
    for (int i = 0; i < 3; ++i) {
        g.rt_hi[i] = rt_hi[i];
        g.rt_lo[i] = rt_lo[i];
    }
    g.rt_chunks[0] = T.wt_chunks;
    g.rt_chunks[1] = g.rt_chunks[2] = T.sk_chunks;
    g.U = U;
    g.ldu = ldu;
    g.perm = perm;
    g.r = r;
    g.pts = T.gen_pts;
    g.dim = T.gen_dim;
    g.dpad = T.gen_dpad;
    g.gen_kind = T.gen_kind;
    g.gen_inv = T.gen_inv;
    g.gen_shift = T.gen_shift;
    return g;
}

template <int MODE, int NMAX, bool GEN>
static void launch_gemm(const TcParams& p, int num_sms, cudaStream_t s) {
    const int grid = std::min(p.ntiles, num_sms);
    tc_gemm_kernel<MODE, NMAX, GEN>
        <<<unsigned(grid), GEN ? kGenThreads : 192, gemm_smem<MODE, NMAX, GEN>(), s>>>(p);
    CUDA_OK(cudaGetLastError());
}

// Cooperative launch: every CTA of the persistent grid is resident at once,
// so tiles waiting on counters bumped by other CTAs always make progress.
template <int MODE, int NMAX, bool GEN>
static void launch_gemm_coop(const TcParams& p, int num_sms, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(std::min(p.ntiles, num_sms)));
    cfg.blockDim = dim3(GEN ? kGenThreads : 192);
    cfg.dynamicSmemBytes = gemm_smem<MODE, NMAX, GEN>();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CUDA_OK(cudaLaunchKernelEx(&cfg, tc_gemm_kernel<MODE, NMAX, GEN>, p));
}

template <bool GEN>
static void launch_gemm_sel(int mode, int piece, const TcParams& p, int num_sms, cudaStream_t s) {
    if (piece <= 128) {
        if (mode == TC_TF32) launch_gemm<TC_TF32, 128, GEN>(p, num_sms, s);
        else if (mode == TC_BF16) launch_gemm<TC_BF16, 128, GEN>(p, num_sms, s);
        else launch_gemm<TC_BF16X3, 128, GEN>(p, num_sms, s);
    } else {
        if (mode == TC_TF32) launch_gemm<TC_TF32, 256, GEN>(p, num_sms, s);
        else if (mode == TC_BF16) launch_gemm<TC_BF16, 256, GEN>(p, num_sms, s);
        else launch_gemm<TC_BF16X3, 256, GEN>(p, num_sms, s);
    }
}

// piece: the tallest task piece among the launch's segments (128 or 256);
// gen: some segment generates its block tiles (the variant with generator warps)
void launch_gemm_mode(int mode, int piece, const TcParams& p, int num_sms, cudaStream_t s, bool gen) {
    if (gen) launch_gemm_sel<true>(mode, piece, p, num_sms, s);
    else launch_gemm_sel<false>(mode, piece, p, num_sms, s);
}

// SM-pair kernel: clusters of two CTAs (static tiles).  The grid is the
// number of clusters the GPU holds at once (pairs of SMs of one GPC), so no
// cluster waits for a second wave.
template <int MODE, int NMAX>
static int resident_pairs(int num_sms) {
    static int cached = 0;  // per kernel instantiation; one device type per process
    if (cached > 0) return cached;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(num_sms / 2 * 2));
    cfg.blockDim = dim3(192);
    cfg.dynamicSmemBytes = Cfg2<MODE, NMAX>::kSmem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    CUDA_OK(cudaOccupancyMaxActiveClusters(&n, tc_gemm_pair_kernel<MODE, NMAX>, &cfg));
    cached = std::max(1, std::min(n, num_sms / 2));
    return cached;
}

static void occupancy_pairs(int num_sms) {
    resident_pairs<TC_TF32, 128>(num_sms);
    resident_pairs<TC_TF32, 256>(num_sms);
    resident_pairs<TC_BF16, 128>(num_sms);
    resident_pairs<TC_BF16, 256>(num_sms);
    resident_pairs<TC_BF16X3, 128>(num_sms);
    resident_pairs<TC_BF16X3, 256>(num_sms);
}

template <int MODE, int NMAX>
static void launch_gemm_pair(const TcParams& p, int num_sms, cudaStream_t s) {
    const int pairs = std::min(p.ntiles, resident_pairs<MODE, NMAX>(num_sms));
    tc_gemm_pair_kernel<MODE, NMAX><<<unsigned(2 * pairs), 192, Cfg2<MODE, NMAX>::kSmem, s>>>(p);
    CUDA_OK(cudaGetLastError());
}

static void launch_gemm_pair_mode(int mode, int piece, const TcParams& p, int num_sms, cudaStream_t s) {
    if (piece <= 128) {
        if (mode == TC_TF32) launch_gemm_pair<TC_TF32, 128>(p, num_sms, s);
        else if (mode == TC_BF16) launch_gemm_pair<TC_BF16, 128>(p, num_sms, s);
        else launch_gemm_pair<TC_BF16X3, 128>(p, num_sms, s);
    } else {
        if (mode == TC_TF32) launch_gemm_pair<TC_TF32, 256>(p, num_sms, s);
        else if (mode == TC_BF16) launch_gemm_pair<TC_BF16, 256>(p, num_sms, s);
        else launch_gemm_pair<TC_BF16X3, 256>(p, num_sms, s);
    }
}

template <bool GEN>
static void launch_gemm_coop_sel(int mode, int piece, const TcParams& p, int num_sms, cudaStream_t s) {
    if (piece <= 128) {
        if (mode == TC_TF32) launch_gemm_coop<TC_TF32, 128, GEN>(p, num_sms, s);
        else if (mode == TC_BF16) launch_gemm_coop<TC_BF16, 128, GEN>(p, num_sms, s);
        else launch_gemm_coop<TC_BF16X3, 128, GEN>(p, num_sms, s);
    } else {
        if (mode == TC_TF32) launch_gemm_coop<TC_TF32, 256, GEN>(p, num_sms, s);
        else if (mode == TC_BF16) launch_gemm_coop<TC_BF16, 256, GEN>(p, num_sms, s);
        else launch_gemm_coop<TC_BF16X3, 256, GEN>(p, num_sms, s);
    }
}

void launch_gemm_coop_mode(int mode, int piece, const TcParams& p, int num_sms, cudaStream_t s, bool gen) {
    if (gen) launch_gemm_coop_sel<true>(mode, piece, p, num_sms, s);
    else launch_gemm_coop_sel<false>(mode, piece, p, num_sms, s);
}

void launch_gather(int mode, const TcPrec& T, const float* W, int64_t ldw, const int64_t* perm,
                          uint8_t* wt_hi, uint8_t* wt_lo, int r, cudaStream_t s) {
    dim3 grid(unsigned(T.wt_chunks), unsigned((r + 127) / 128));
    if (mode == TC_TF32)
        tc_gather_kernel<TC_TF32><<<grid, 256, 0, s>>>(W, ldw, perm, T.d_chunk_pos, T.d_chunk_valid, wt_hi, wt_lo,
                                                       T.wt_chunks, r);
    else if (mode == TC_BF16)
        tc_gather_kernel<TC_BF16><<<grid, 256, 0, s>>>(W, ldw, perm, T.d_chunk_pos, T.d_chunk_valid, wt_hi, wt_lo,
                                                       T.wt_chunks, r);
    else
        tc_gather_kernel<TC_BF16X3><<<grid, 256, 0, s>>>(W, ldw, perm, T.d_chunk_pos, T.d_chunk_valid, wt_hi,
                                                         wt_lo, T.wt_chunks, r);
    CUDA_OK(cudaGetLastError());
}

static int tc_launch_all(Handle& H, DeviceState& D, TcPrec& T, const float* W, int64_t ldw, float* U, int64_t ldu,
                         int r, cudaStream_t s) {
    const int n_rtiles = (r + 127) / 128;
    int launches = 0;
    const bool timing = H.timing != 0 && D.ev_ok;
    if (timing) CUDA_OK(cudaEventRecord(D.ev[0], s));
    launch_gather(T.mode, T, W, ldw, D.d_idx, T.rt_hi[0], T.rt_lo[0], r, s);
    ++launches;
    if (timing) CUDA_OK(cudaEventRecord(D.ev[1], s));
    TcParams p{};
    p.nsegs = 1;
    p.err = T.d_err;
    const int sched = H.tc_schedule[T.mode];
    if (sched == GOFMM_SCHED_PAIR && T.gen)
        fail(GOFMM_ERR_UNSUPPORTED, "the SM-pair schedule needs cached K blocks (GOFMM_CACHE_BLOCKS)");
    // one dependency-driven launch of the tasks of plan F
    auto run_fused = [&](TcFused& F) {
        if (F.tasks.empty()) return;
        if (F.counters_nrt < n_rtiles) fail(GOFMM_ERR_ARG, "fused plan not prepared for this r");
        CUDA_OK(cudaMemsetAsync(F.d_counters, 0, (size_t(F.ncounters) * n_rtiles + 1) * sizeof(int), s));
        TcParams q{};
        q.nsegs = 1;
        q.err = T.d_err;
        if (H.tc_order[T.mode] == GOFMM_ORDER_READY) {
            // list part and queued part; the queue and the pending counts
            // start from their initial copies
            TcFused::Ready& R = ready_tiles(F, n_rtiles);
            CUDA_OK(cudaMemcpyAsync(R.queue, R.queue0, size_t(2 + R.n) * sizeof(int), cudaMemcpyDeviceToDevice, s));
            if (R.n) CUDA_OK(cudaMemcpyAsync(R.pending, R.pending0, size_t(R.n) * sizeof(int), cudaMemcpyDeviceToDevice, s));
            q.tiles = R.tiles;
            q.ntiles = R.n_static + R.n;
            q.ready = TcReady{R.queue, R.pending, R.cons_off, R.cons, R.req, R.n_static, R.n};
        } else {
            const auto tl = fused_tiles(F, n_rtiles, H.tc_order[T.mode]);
            q.tiles = tl.first;
            q.ntiles = tl.second;
        }
        TcSeg g = make_seg(T, T.launches.front(), T.rt_hi, T.rt_lo, U, ldu, D.d_idx, r);
        g.tasks = F.d_tasks;
        g.slabs = F.d_slabs;
        g.dep_off = F.d_dep_off;
        g.deps = F.d_deps;
        if (F.stall_next) {  // diagnostic: one dependency nothing satisfies
            if (F.d_slabs_stall) g.slabs = F.d_slabs_stall;
            else g.deps = F.d_deps_stall;
            F.stall_next = false;
        }
        g.sig = F.d_sig;
        g.counters = F.d_counters;
        g.dep_nrt = n_rtiles;
        q.tile_next = F.d_counters + size_t(F.ncounters) * n_rtiles;
        q.segs[0] = g;
        launch_gemm_coop_mode(T.mode, T.piece, q, T.num_sms, s, T.gen);
        ++launches;
    };
    if (H.timing != 1 && sched == GOFMM_SCHED_HYBRID) {
        // upward pass in one dependency-driven launch, S2S in one launch,
        // downward pass and leaves in one dependency-driven launch
        D.last_fused = false;
        run_fused(T.fused_up);
        if (timing) CUDA_OK(cudaEventRecord(D.ev[2], s));
        CUDA_OK(cudaMemsetAsync(T.d_claims, 0, kClaimSlots * sizeof(int), s));
        int claim = 0;
        for (TcLaunch& l : T.launches) {
            if (l.stage != 2 || l.tasks.empty()) continue;
            const auto tl = launch_tiles(l, n_rtiles, H.tc_order[T.mode], false, l.wmax);
            p.tiles = tl.first;
            p.ntiles = tl.second;
            p.segs[0] = make_seg(T, l, T.rt_hi, T.rt_lo, U, ldu, D.d_idx, r);
            p.tile_next = claim < kClaimSlots ? T.d_claims + claim++ : nullptr;  // dynamic claiming
            launch_gemm_mode(T.mode, T.piece, p, T.num_sms, s, T.gen);
            ++launches;
        }
        p.tile_next = nullptr;
        if (timing) CUDA_OK(cudaEventRecord(D.ev[3], s));
        run_fused(T.fused_down);
        if (timing)
            for (int i = 4; i <= 5; ++i) CUDA_OK(cudaEventRecord(D.ev[i], s));
    } else if (H.timing == 1 || sched != GOFMM_SCHED_FUSED) {
        // one launch per stage (stage timing, or a staged schedule)
        D.last_fused = false;
        const bool pair = sched == GOFMM_SCHED_PAIR;
        int stage_done = 1;
        if (!pair) CUDA_OK(cudaMemsetAsync(T.d_claims, 0, kClaimSlots * sizeof(int), s));
        int claim = 0;
        for (TcLaunch& l : T.launches) {
            while (stage_done < l.stage) CUDA_OK(cudaEventRecord(D.ev[++stage_done], s));
            if (l.tasks.empty()) continue;
            const auto tl = launch_tiles(l, n_rtiles, H.tc_order[T.mode], pair, pair ? 2 : l.wmax);
            p.tiles = tl.first;
            p.ntiles = tl.second;
            p.segs[0] = make_seg(T, l, T.rt_hi, T.rt_lo, U, ldu, D.d_idx, r);
            // the SM-pair kernel splits its tiles statically; the single-SM
            // kernel claims them from a counter (no stragglers at the end)
            p.tile_next = !pair && claim < kClaimSlots ? T.d_claims + claim++ : nullptr;
            if (pair) launch_gemm_pair_mode(T.mode, T.piece, p, T.num_sms, s);
            else launch_gemm_mode(T.mode, T.piece, p, T.num_sms, s, T.gen);
            ++launches;
        }
        p.tile_next = nullptr;
        while (stage_done < 5) CUDA_OK(cudaEventRecord(D.ev[++stage_done], s));
    } else {
        // every grouped GEMM in one dependency-driven launch
        D.last_fused = true;
        run_fused(T.fused);
        if (timing)
            for (int i = 2; i <= 5; ++i) CUDA_OK(cudaEventRecord(D.ev[i], s));
    }
    CUDA_OK(cudaMemcpyAsync(T.h_err, T.d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    return launches;
}

int tc_run(Handle& H, DeviceState& D, const float* W, int64_t ldw, float* U, int64_t ldu, int r, int precision,
           cudaStream_t s) {
    TcPrec& T = *D.tc->prec[mode_of(precision)];
    if (*reinterpret_cast<volatile int*>(T.h_err) != 0)
        fail(GOFMM_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait (code " + std::to_string(*T.h_err) + ")");
    return tc_launch_all(H, D, T, W, ldw, U, ldu, r, s);
}

void tc_stall_next(DeviceState& D, int precision) {
    if (!D.tc || !D.tc->prec[mode_of(precision)])
        fail(GOFMM_ERR_ARG, "handle not prepared for this precision: call gofmm_prepare first");
    TcFused& F = D.tc->prec[mode_of(precision)]->fused;
    if (!F.d_deps_stall && !F.d_slabs_stall) {
        // one dependency of the plan gets an arrival count no counter reaches:
        // a slab's operand dependency, else a task's
        std::vector<TcSlab> slabs(F.slabs);
        bool done = false;
        for (TcSlab& sl : slabs)
            if (sl.dep_c0 >= 0) {
                sl.dep_n0 = 1 << 30;
                done = true;
                break;
            }
        if (done) {
            F.d_slabs_stall = dupload(slabs);
        } else {
            std::vector<int32_t> deps(F.deps_host);
            if (deps.size() < 2) fail(GOFMM_ERR_UNSUPPORTED, "the plan has no dependency to stall");
            deps[1] = 1 << 30;
            F.d_deps_stall = dupload(deps);
        }
    }
    F.stall_next = true;
}

void tc_clear_error(DeviceState& D) {
    if (!D.tc) return;
    for (TcPrec* T : D.tc->prec)
        if (T && T->h_err && *T->h_err) {
            CUDA_OK(cudaMemset(T->d_err, 0, sizeof(int)));
            *T->h_err = 0;
        }
}

int tc_error(const DeviceState& D) {
    if (!D.tc) return 0;
    for (const TcPrec* T : D.tc->prec)
        if (T && T->h_err && *T->h_err) return *T->h_err;
    return 0;
}

static void free_prec(TcPrec*& T) {
    if (!T) return;
    {
        for (TcLaunch& l : T->launches) {
            dfree(l.d_tasks);
            dfree(l.d_slabs);
            for (auto& kv : l.tiles) dfree(kv.second.first);
        }
        dfree(T->d_chunk_pos); dfree(T->d_chunk_valid); dfree(T->b_hi); dfree(T->b_lo); dfree(T->d_err); dfree(T->d_claims);
        dfree(T->gen_pts);
        for (TcFused* F : {&T->fused, &T->fused_up, &T->fused_down}) {
            dfree(F->d_tasks); dfree(F->d_slabs); dfree(F->d_dep_off); dfree(F->d_deps); dfree(F->d_sig);
            dfree(F->d_deps_stall);
            dfree(F->d_slabs_stall);
            dfree(F->d_counters);
            for (auto& kv : F->tiles) dfree(kv.second.first);
            for (auto& kv : F->ready) {
                TcFused::Ready& R = kv.second;
                dfree(R.tiles); dfree(R.queue); dfree(R.queue0); dfree(R.pending); dfree(R.pending0);
                dfree(R.cons_off); dfree(R.cons); dfree(R.req);
            }
        }
        for (int i = 0; i < 3; ++i) { dfree(T->rt_hi[i]); dfree(T->rt_lo[i]); }
        if (T->h_err) cudaFreeHost(T->h_err);
        delete T;
        T = nullptr;
    }
}

void tc_drop_plan(DeviceState& D, int precision) {
    if (!D.tc) return;
    CUDA_OK(cudaDeviceSynchronize());  // no launch may still read the plan
    free_prec(D.tc->prec[mode_of(precision)]);
}

void tc_destroy(DeviceState& D) {
    if (!D.tc) return;
    for (TcPrec*& T : D.tc->prec) free_prec(T);
    delete D.tc;
    D.tc = nullptr;
}

}  // namespace gofmm
