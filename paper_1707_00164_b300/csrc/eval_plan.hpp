// Evaluation plan shared by the host planner and the device kernels.
//
// Every stage of Alg. 7 is a *grouped GEMM*: a list of tasks, each writing
// an m x r block of one output buffer as a sum over "slabs"
//     out[task rows] = sum_slab  A_slab (m x k) * B_slab (k x r),
// where A_slab is a cached K block, an interpolation matrix P / P^T, or K
// entries generated on the fly, and B_slab is a row range of one of the
// tree-ordered right-hand-side buffers.  The tasks of one launch write
// disjoint rows (of one of the output buffers, chosen per task), so no
// launch accumulates into memory another CTA writes.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define GOFMM_HD __host__ __device__
#else
#define GOFMM_HD
#endif

namespace gofmm {

enum ASrc : int32_t { A_KSTORE = 0, A_PSTORE = 1, A_GEN = 2 };
enum BSrc : int32_t { B_WT = 0, B_WTIL = 1, B_UTIL = 2 };
enum OutBuf : int32_t { OUT_WTIL = 0, OUT_UTIL = 1, OUT_U = 2 };

struct Slab {
    int64_t a_off;  // KSTORE/PSTORE: element offset of A; GEN: offset of the row index list in idx[]
    int64_t a_col;  // GEN: offset of the column index list in idx[]
    int64_t b_row;  // first row of B in its buffer
    int32_t k;      // inner dimension
    int32_t lda;    // KSTORE/PSTORE: leading dimension of A (row-major)
    int32_t a_src;  // ASrc
    int32_t b_src;  // BSrc
};

struct Task {
    int64_t out_row;  // first output row (tree position for OUT_U, packed row otherwise)
    int32_t m;        // rows
    int32_t slab0, slab1;  // slabs [slab0, slab1)
    int32_t flags;    // bits 0-3: OutBuf; bit 4: accumulate (out += sum of slabs)
};
constexpr int32_t kTaskAccumulate = 16;
GOFMM_HD inline int32_t task_out(int32_t flags) { return flags & 15; }
GOFMM_HD inline bool task_accumulate(int32_t flags) { return (flags & kTaskAccumulate) != 0; }

struct Tile {
    int32_t task;
    int32_t m0;  // first row of this tile inside the task
};

// Cached K block to be generated on the device (row-major dst).
struct GenBlock {
    int64_t dst;
    int64_t roff, coff;  // offsets of the row / column index lists in idx[]
    int32_t nr, nc;
};

}  // namespace gofmm
