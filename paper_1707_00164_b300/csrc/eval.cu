// Device side of the GOFMM evaluation U = K~ W (Alg. 7, Table 2) on one GPU.
//
// Launch sequence of one evaluation (all on the caller's stream):
//   stage 0  gather W (original order) into tree order WT       (step a0)
//   stage 1  leaf N2S tasks  w~_b = P_{b~b} WT[b], then one grouped launch
//            per inner level, bottom-up:
//            w~_a = P_{a~[l~r~]} [w~_l; w~_r]                  (N2S, POST)
//   stage 2  one grouped launch over all levels:
//            u~_b = sum_{a in Far(b)} K_{b~a~} w~_a            (S2S)
//   stage 3  one launch per level, top-down, accumulating in place
//            u~_b += (P^T_{p~[l~r~]} u~_p)[rows of b]          (S2N, PRE)
//   stage 4  one grouped launch over the leaves, scattered to the original
//            order:  U[b] = P^T_{b~b} u~_b + sum_{a in Near(b)} K_{ba} WT[a]
//                                                              (S2N leaf + L2L)
// Every launch is a grouped GEMM (eval_plan.hpp) whose tasks own disjoint
// output rows; the sum over slabs runs in a fixed order inside one CTA, so
// results are deterministic and nothing is accumulated with atomics (the
// in-place S2N pushes read and write only rows their own thread owns).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>

#include "eval_plan.hpp"
#include "eval_state.hpp"
#include "eval_tc.hpp"

namespace gofmm {

// ------------------------------------------------------------- kernels --
namespace {

// WT[i, :] = W[perm[i], :]  (step a0: tree-order gather)
template <typename T>
__global__ void gather_rows_kernel(const T* __restrict__ W, int64_t ldw, const int64_t* __restrict__ perm,
                                   T* __restrict__ WT, int64_t n, int r) {
    const int64_t row = int64_t(blockIdx.x) * blockDim.y + threadIdx.y;
    if (row >= n) return;
    const T* src = W + perm[row] * ldw;
    T* dst = WT + row * int64_t(r);
    for (int c = threadIdx.x; c < r; c += blockDim.x) dst[c] = src[c];
}

// Cached K blocks generated from the points in FP64 (Kba / SKba caching of
// Alg. 2 steps 10-11, done on the device for generator matrices).
template <typename T>
__global__ void gen_blocks_kernel(const GenBlock* __restrict__ blks, const int64_t* __restrict__ idx,
                                  const double* __restrict__ pts, int dim, int kind, double h, double shift,
                                  T* __restrict__ dst) {
    const GenBlock b = blks[blockIdx.x];
    const int64_t total = int64_t(b.nr) * b.nc;
    const double two_h2 = 2.0 * h * h, h2 = h * h;
    for (int64_t e = int64_t(blockIdx.y) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.y) * blockDim.x) {
        const int i = int(e / b.nc), j = int(e % b.nc);
        const int64_t ri = idx[b.roff + i], cj = idx[b.coff + j];
        double acc = 0.0;
        for (int d = 0; d < dim; ++d) {
            const double t = pts[ri * dim + d] - pts[cj * dim + d];
            acc += t * t;
        }
        double v = kind == GOFMM_GEN_GAUSSIAN ? exp(-(acc / two_h2)) : 1.0 / sqrt(1.0 + acc / h2);
        if (ri == cj) v += shift;
        dst[b.dst + e] = T(v);
    }
}

template <typename T>
struct GemmParams {
    const Task* tasks;
    const Tile* tiles;
    const Slab* slabs;
    const T* kstore;
    const T* pstore;
    const T* b0;
    const T* b1;
    const T* b2;
    int64_t ldb;
    const int64_t* idx;
    const T* pts;
    int dim, gen_kind;
    T gen_inv, gen_shift;  // Gaussian: exp(-d2*inv), inv = 1/(2h^2); IMQ: rsqrt(1 + d2*inv), inv = 1/h^2
    T* out_wtil;  // OUT_WTIL / OUT_UTIL: packed rows, leading dimension r
    T* out_util;
    T* out_u;     // OUT_U: the caller's U, rows through the tree permutation
    int64_t ldu;
    const int64_t* perm;
    int r;
};

__device__ __forceinline__ double kexp(double x) { return exp(x); }
__device__ __forceinline__ float kexp(float x) { return expf(x); }
__device__ __forceinline__ double krsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float krsqrt(float x) { return rsqrtf(x); }

// Kernel entry K(i, j) generated in the working precision (fused sampling).
template <typename T>
__device__ __forceinline__ T gen_entry(const GemmParams<T>& p, int64_t ri, int64_t cj) {
    T acc = T(0);
    for (int d = 0; d < p.dim; ++d) {
        const T t = p.pts[ri * p.dim + d] - p.pts[cj * p.dim + d];
        acc += t * t;
    }
    T v = p.gen_kind == GOFMM_GEN_GAUSSIAN ? kexp(-acc * p.gen_inv) : krsqrt(T(1) + acc * p.gen_inv);
    if (ri == cj) v += p.gen_shift;
    return v;
}

// Grouped GEMM on CUDA cores (FP64 parity mode and the plain FP32 mode).
// CTA tile BM x BN = (16 TM) x (16 TN), 256 threads (two CTAs per SM), each
// owning TM x TN outputs split in two halves of the tile for conflict-free
// shared reads.  The K loop runs over all chunks of all slabs of the task;
// the next chunk is loaded into registers while the current one is
// multiplied from the other half of a double-buffered shared tile.
template <typename T, int TM, int TN>
__global__ void __launch_bounds__(256, 2) gemm_simt_kernel(const GemmParams<T> p) {
    constexpr int BM = 16 * TM, BN = 16 * TN, BK = 8;
    constexpr int AE = BM * BK / 256, BE = BK * BN / 256;  // elements per thread and chunk
    constexpr int APAD = BM + 8;                             // padded A rows: fewer bank conflicts
    __shared__ __align__(16) T As[2][BK][APAD];
    __shared__ __align__(16) T Bs[2][BK][BN];
    const Tile tl = p.tiles[blockIdx.x];
    const Task tk = p.tasks[tl.task];
    const int m0 = tl.m0;
    const int n0 = blockIdx.y * BN;
    const int mrows = min(BM, tk.m - m0);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    T ra[AE], rb[BE];
    // load chunk (slab sl, rows k0..k0+BK) into registers
    auto load = [&](const Slab& sl, int k0) {
        const T* bptr = (sl.b_src == B_WT ? p.b0 : sl.b_src == B_WTIL ? p.b1 : p.b2) + sl.b_row * p.ldb;
        const T* aptr = (sl.a_src == A_KSTORE ? p.kstore : p.pstore) + sl.a_off;
#pragma unroll
        for (int u = 0; u < AE; ++u) {
            const int e = tid + u * 256, mm = e / BK, kk = e % BK;
            T v = T(0);
            if (mm < mrows && k0 + kk < sl.k) {
                if (sl.a_src == A_GEN)
                    v = gen_entry(p, p.idx[sl.a_off + m0 + mm], p.idx[sl.a_col + k0 + kk]);
                else
                    v = aptr[int64_t(m0 + mm) * sl.lda + k0 + kk];
            }
            ra[u] = v;
        }
#pragma unroll
        for (int u = 0; u < BE; ++u) {
            const int e = tid + u * 256, kk = e / BN, nn = e % BN;
            rb[u] = (k0 + kk < sl.k && n0 + nn < p.r) ? bptr[int64_t(k0 + kk) * p.ldb + n0 + nn] : T(0);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int u = 0; u < AE; ++u) {
            const int e = tid + u * 256;
            As[buf][e % BK][e / BK] = ra[u];
        }
#pragma unroll
        for (int u = 0; u < BE; ++u) {
            const int e = tid + u * 256;
            Bs[buf][e / BN][e % BN] = rb[u];
        }
    };

    // first non-empty chunk
    int si = tk.slab0, k0 = 0;
    while (si < tk.slab1 && p.slabs[si].k <= 0) ++si;
    Slab cur{};
    if (si < tk.slab1) {
        cur = p.slabs[si];
        load(cur, 0);
        store(0);
    }
    __syncthreads();
    int buf = 0;
    while (si < tk.slab1) {
        // position of the next chunk
        int nsi = si, nk0 = k0 + BK;
        Slab nxt = cur;
        if (nk0 >= cur.k) {
            nk0 = 0;
            ++nsi;
            while (nsi < tk.slab1 && p.slabs[nsi].k <= 0) ++nsi;
            if (nsi < tk.slab1) nxt = p.slabs[nsi];
        }
        const bool more = nsi < tk.slab1;
        if (more) load(nxt, nk0);  // in flight while the current chunk is multiplied
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i)
                a[i] = As[buf][kk][i < TM / 2 ? ty * (TM / 2) + i : BM / 2 + ty * (TM / 2) + i - TM / 2];
#pragma unroll
            for (int j = 0; j < TN; ++j)
                b[j] = Bs[buf][kk][j < TN / 2 ? tx * (TN / 2) + j : BN / 2 + tx * (TN / 2) + j - TN / 2];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
        si = nsi;
        k0 = nk0;
        cur = nxt;
    }
    const int okind = task_out(tk.flags);
    const bool accum = task_accumulate(tk.flags);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int row = i < TM / 2 ? ty * (TM / 2) + i : BM / 2 + ty * (TM / 2) + i - TM / 2;
        if (row >= mrows) continue;
        const int64_t orow = tk.out_row + m0 + row;
        T* o = okind == OUT_U ? p.out_u + p.perm[orow] * p.ldu
                              : (okind == OUT_WTIL ? p.out_wtil : p.out_util) + orow * int64_t(p.r);
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int col = n0 + (j < TN / 2 ? tx * (TN / 2) + j : BN / 2 + tx * (TN / 2) + j - TN / 2);
            if (col < p.r) o[col] = accum ? o[col] + acc[i][j] : acc[i][j];
        }
    }
}

}  // namespace

static void build_plan(const Structure& st, bool cached, DeviceState& D) {
    const int64_t nn = st.n_nodes(), nl = st.n_leaves(), N = st.n;
    const int L = st.depth;
    D.n = N;
    D.skel_off.assign(nn, -1);
    int64_t S = 0;
    for (int64_t h = 1; h < nn; ++h) { D.skel_off[h] = S; S += int64_t(st.skel[h].size()); }
    D.S_tot = S;
    D.idx = st.perm;
    for (int64_t h = 1; h < nn; ++h) D.idx.insert(D.idx.end(), st.skel[h].begin(), st.skel[h].end());
    // P-store: P_h (s x ncols) then P_h^T (ncols x s)
    D.p_off.assign(nn, -1);
    D.pt_off.assign(nn, -1);
    D.pstore_host.clear();
    for (int64_t h = 1; h < nn; ++h) {
        const int64_t s = int64_t(st.skel[h].size()), nc = st.ncols(h);
        D.p_off[h] = int64_t(D.pstore_host.size());
        D.pstore_host.insert(D.pstore_host.end(), st.P[h].begin(), st.P[h].end());
        D.pt_off[h] = int64_t(D.pstore_host.size());
        for (int64_t c = 0; c < nc; ++c)
            for (int64_t t = 0; t < s; ++t) D.pstore_host.push_back(st.P[h][size_t(t * nc + c)]);
    }
    D.pstore_elems = int64_t(D.pstore_host.size());
    // K-store layout
    D.kblocks.clear();
    std::vector<std::vector<int64_t>> near_koff(nl), far_koff(nn);
    int64_t K = 0;
    for (int64_t b = 0; b < nl; ++b) {
        const int64_t hb = st.leaf_node(b);
        for (int64_t a : st.near[b]) {
            const int64_t ha = st.leaf_node(a);
            near_koff[b].push_back(K);
            D.kblocks.push_back(GenBlock{K, st.node_off[hb], st.node_off[ha], int32_t(st.node_size[hb]),
                                         int32_t(st.node_size[ha])});
            K += st.node_size[hb] * st.node_size[ha];
        }
    }
    for (int64_t h = 1; h < nn; ++h)
        for (int64_t a : st.far[h]) {
            far_koff[h].push_back(K);
            const int64_t sh = int64_t(st.skel[h].size()), sa = int64_t(st.skel[a].size());
            D.kblocks.push_back(GenBlock{K, N + D.skel_off[h], N + D.skel_off[a], int32_t(sh), int32_t(sa)});
            K += sh * sa;
        }
    D.kstore_elems = cached ? K : 0;

    // u~ is identically zero below nodes with no far field on the path to
    // the root; those tasks and the push slabs reading them are skipped.
    std::vector<char> field(nn, 0);
    for (int64_t h = 1; h < nn; ++h) field[h] = !st.far[h].empty() || (h > 0 && field[(h - 1) / 2]);

    D.launches.clear();
    auto add_launch = [&](int stage) -> Launch& {
        D.launches.emplace_back();
        D.launches.back().stage = stage;
        return D.launches.back();
    };
    auto slab = [](int a_src, int64_t a_off, int64_t a_col, int lda, int k, int b_src, int64_t b_row) {
        Slab s;
        s.a_off = a_off; s.a_col = a_col; s.b_row = b_row; s.k = k; s.lda = lda; s.a_src = a_src; s.b_src = b_src;
        return s;
    };
    if (L == 0) {
        // a single leaf: U = K W
        Launch& lo = add_launch(4);
        Task t{0, int32_t(N), 0, 0, OUT_U};
        lo.slabs.push_back(cached ? slab(A_KSTORE, 0, 0, int(N), int(N), B_WT, 0)
                                  : slab(A_GEN, 0, 0, 0, int(N), B_WT, 0));
        t.slab1 = 1;
        lo.tasks.push_back(t);
        return;
    }
    // stage 1 (upward): leaf N2S, then inner N2S bottom-up
    {
        Launch& l = add_launch(1);
        for (int64_t b = 0; b < nl; ++b) {
            const int64_t h = st.leaf_node(b);
            Task t{D.skel_off[h], int32_t(st.skel[h].size()), int32_t(l.slabs.size()), 0, OUT_WTIL};
            l.slabs.push_back(slab(A_PSTORE, D.p_off[h], 0, int(st.node_size[h]), int(st.node_size[h]), B_WT,
                                   st.node_off[h]));
            t.slab1 = int32_t(l.slabs.size());
            l.tasks.push_back(t);
        }
    }
    for (int lvl = L - 1; lvl >= 1; --lvl) {
        Launch& l = add_launch(1);
        for (int64_t h = (int64_t(1) << lvl) - 1; h < (int64_t(2) << lvl) - 1; ++h) {
            const int nc = int(st.ncols(h));
            Task t{D.skel_off[h], int32_t(st.skel[h].size()), int32_t(l.slabs.size()), 0, OUT_WTIL};
            l.slabs.push_back(slab(A_PSTORE, D.p_off[h], 0, nc, nc, B_WTIL, D.skel_off[2 * h + 1]));
            t.slab1 = int32_t(l.slabs.size());
            l.tasks.push_back(t);
        }
    }
    // stage 2: S2S for every node with a field, all levels in one launch
    // (tasks of every level run side by side, heaviest first) ...
    {
        Launch& l = add_launch(2);
        for (int64_t h = 1; h < nn; ++h) {
            if (!field[h]) continue;
            const int64_t sh = int64_t(st.skel[h].size());
            Task t{D.skel_off[h], int32_t(sh), int32_t(l.slabs.size()), 0, OUT_UTIL};
            for (size_t u = 0; u < st.far[h].size(); ++u) {
                const int64_t a = st.far[h][u];
                const int sa = int(st.skel[a].size());
                l.slabs.push_back(cached ? slab(A_KSTORE, far_koff[h][u], 0, sa, sa, B_WTIL, D.skel_off[a])
                                         : slab(A_GEN, N + D.skel_off[h], N + D.skel_off[a], 0, sa, B_WTIL,
                                                D.skel_off[a]));
            }
            t.slab1 = int32_t(l.slabs.size());
            l.tasks.push_back(t);
        }
        if (l.tasks.empty()) D.launches.pop_back();
    }
    // ... then the S2N pushes level by level, top-down, accumulated in place:
    // u~_h += (P^T_{p~[l~r~]} u~_p)[rows of h]
    for (int lvl = 2; lvl <= L; ++lvl) {
        Launch& l = add_launch(3);
        for (int64_t h = (int64_t(1) << lvl) - 1; h < (int64_t(2) << lvl) - 1; ++h) {
            const int64_t p = (h - 1) / 2;
            if (!field[p]) continue;
            const int sp = int(st.skel[p].size());
            const int64_t rowoff = (h == 2 * p + 1) ? 0 : int64_t(st.skel[2 * p + 1].size());
            Task t{D.skel_off[h], int32_t(st.skel[h].size()), int32_t(l.slabs.size()), 0,
                   OUT_UTIL | kTaskAccumulate};
            l.slabs.push_back(slab(A_PSTORE, D.pt_off[p] + rowoff * sp, 0, sp, sp, B_UTIL, D.skel_off[p]));
            t.slab1 = int32_t(l.slabs.size());
            l.tasks.push_back(t);
        }
        if (l.tasks.empty()) D.launches.pop_back();
    }
    // stage 4: leaf S2N + L2L, scattered to the original order
    {
        Launch& l = add_launch(4);
        for (int64_t b = 0; b < nl; ++b) {
            const int64_t h = st.leaf_node(b);
            Task t{st.node_off[h], int32_t(st.node_size[h]), int32_t(l.slabs.size()), 0, OUT_U};
            for (size_t u = 0; u < st.near[b].size(); ++u) {
                const int64_t ha = st.leaf_node(st.near[b][u]);
                const int na = int(st.node_size[ha]);
                l.slabs.push_back(cached ? slab(A_KSTORE, near_koff[b][u], 0, na, na, B_WT, st.node_off[ha])
                                         : slab(A_GEN, st.node_off[h], st.node_off[ha], 0, na, B_WT,
                                                st.node_off[ha]));
            }
            if (field[h]) {
                const int sh = int(st.skel[h].size());
                l.slabs.push_back(slab(A_PSTORE, D.pt_off[h], 0, sh, sh, B_UTIL, D.skel_off[h]));
            }
            t.slab1 = int32_t(l.slabs.size());
            l.tasks.push_back(t);
        }
    }
    // heaviest tasks first inside every launch (better tail behaviour)
    for (Launch& l : D.launches) {
        std::vector<int64_t> work(l.tasks.size());
        for (size_t i = 0; i < l.tasks.size(); ++i) {
            int64_t k = 0;
            for (int s = l.tasks[i].slab0; s < l.tasks[i].slab1; ++s) k += l.slabs[s].k;
            work[i] = k * l.tasks[i].m;
        }
        std::vector<size_t> o(l.tasks.size());
        for (size_t i = 0; i < o.size(); ++i) o[i] = i;
        std::stable_sort(o.begin(), o.end(), [&](size_t a, size_t b) { return work[a] > work[b]; });
        std::vector<Task> t2;
        for (size_t i : o) t2.push_back(l.tasks[i]);
        l.tasks = t2;
    }
}

std::pair<Tile*, int> tiles_for(Launch& l, int bm) {
    auto it = l.tiles.find(bm);
    if (it != l.tiles.end()) return it->second;
    std::vector<Tile> t;
    for (size_t i = 0; i < l.tasks.size(); ++i)
        for (int m0 = 0; m0 < std::max(l.tasks[i].m, 1); m0 += bm) t.push_back(Tile{int32_t(i), m0});
    auto v = std::make_pair(dupload(t), int(t.size()));
    l.tiles[bm] = v;
    return v;
}

static void ensure_base(Handle& H) {
    if (H.dev) return;
    const Structure& st = H.st;
    const bool cached = st.prm.cache_mode == GOFMM_CACHE_BLOCKS;
    auto D = std::make_unique<DeviceState>();
    D->device = st.prm.device;
    build_plan(st, cached, *D);
    D->d_idx = dupload(D->idx);
    for (Launch& l : D->launches) {
        l.d_tasks = dupload(l.tasks);
        l.d_slabs = dupload(l.slabs);
    }
    D->d_kblocks = dupload(D->kblocks);
    if (H.K.is_generator()) {
        D->d_pts64 = dupload(H.K.pts);
        std::vector<float> p32(H.K.pts.begin(), H.K.pts.end());
        D->d_pts32 = dupload(p32);
    }
    for (int i = 0; i < 6; ++i) CUDA_OK(cudaEventCreate(&D->ev[i]));
    D->ev_ok = true;
    CUDA_OK(cudaStreamCreateWithFlags(&D->capture_stream, cudaStreamNonBlocking));
    H.dev = D.release();
}

template <typename T>
static void ensure_stores(Handle& H, int fi) {
    DeviceState& D = *H.dev;
    Family& F = D.fam[fi];
    if (F.stores) return;
    const Structure& st = H.st;
    std::vector<T> ps(D.pstore_host.begin(), D.pstore_host.end());
    F.pstore = dupload(ps);
    if (D.kstore_elems > 0) {
        T* ks = dalloc<T>(size_t(D.kstore_elems));
        F.kstore = ks;
        if (H.K.is_generator()) {
            if (!D.kblocks.empty()) {
                dim3 grid(unsigned(D.kblocks.size()), 8);
                gen_blocks_kernel<T><<<grid, 256>>>(D.d_kblocks, D.d_idx, D.d_pts64, H.K.dim, H.K.kind, H.K.h,
                                                    H.K.shift, ks);
                CUDA_OK(cudaGetLastError());
            }
        } else {
            std::vector<T> host(size_t(D.kstore_elems));
            size_t pos = 0;
            for (const auto& lst : st.near_blocks)
                for (const auto& blk : lst)
                    for (double v : blk) host[pos++] = T(v);
            for (const auto& lst : st.far_blocks)
                for (const auto& blk : lst)
                    for (double v : blk) host[pos++] = T(v);
            if (int64_t(pos) != D.kstore_elems) fail(GOFMM_ERR_ARG, "cached blocks do not match the plan");
            CUDA_OK(cudaMemcpy(ks, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice));
        }
        CUDA_OK(cudaDeviceSynchronize());
    }
    F.stores = true;
}

template <typename T>
static void ensure_workspace(Handle& H, int fi, int64_t r) {
    DeviceState& D = *H.dev;
    Family& F = D.fam[fi];
    if (F.ws_r >= r) return;
    dfree(F.WT); dfree(F.WTIL); dfree(F.UTIL);
    F.WT = F.WTIL = F.UTIL = nullptr;
    for (int k = 0; k < Family::kStageSlots; ++k) {  // staging too, so it is sized again
        dfree(F.sW[k]);
        dfree(F.sU[k]);
        F.sW[k] = F.sU[k] = nullptr;
    }
    F.ws_r = 0;
    F.WT = dalloc<T>(size_t(D.n * r));
    F.WTIL = dalloc<T>(size_t(std::max<int64_t>(D.S_tot, 1) * r));
    F.UTIL = dalloc<T>(size_t(std::max<int64_t>(D.S_tot, 1) * r));
    F.ws_r = r;
}

template <typename T>
static void ensure_staging(Handle& H, int fi, int64_t r, bool all) {
    Family& F = H.dev->fam[fi];
    const int want = all ? Family::kStageSlots : 1;
    bool have = F.stage_r >= r;
    for (int k = 0; k < want; ++k) have = have && F.sW[k];
    if (have) return;
    // buffers still read or written by earlier asynchronous calls
    CUDA_OK(cudaDeviceSynchronize());
    const int64_t rr = std::max(r, F.stage_r);
    for (int k = 0; k < Family::kStageSlots; ++k) {
        dfree(F.sW[k]);
        dfree(F.sU[k]);
        F.sW[k] = F.sU[k] = nullptr;
    }
    F.stage_r = 0;
    for (int k = 0; k < want; ++k) {
        F.sW[k] = dalloc<T>(size_t(H.dev->n * rr));
        F.sU[k] = dalloc<T>(size_t(H.dev->n * rr));
    }
    F.stage_r = rr;
    for (cudaEvent_t& e : F.slot_free)
        if (!e) CUDA_OK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
}

static int family_of(int precision) { return precision == GOFMM_PREC_FP64 ? 0 : 1; }

// Column chunks of the copy / compute pipeline of host-buffer evaluations:
// two chunks of whole 128-column r-tiles (more chunks re-read every cached
// block once per chunk, which costs more than the overlap gains).
constexpr int64_t kHostChunk = 128;
static int64_t host_chunk(int64_t r) { return (r / 2 + kHostChunk - 1) / kHostChunk * kHostChunk; }

static void clear_graphs(DeviceState& D) {
    for (auto& kv : D.graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    D.graphs.clear();
}

void device_prepare(Handle& H, int64_t r_max, int precision) {
    if (r_max < 1) fail(GOFMM_ERR_ARG, "r_max must be >= 1");
    if (precision < GOFMM_PREC_FP64 || precision > GOFMM_PREC_BF16X3) fail(GOFMM_ERR_ARG, "unknown precision");
    DeviceGuard g(H.st.prm.device);
    ensure_base(H);
    clear_graphs(*H.dev);  // buffers may move below
    // tile lists of the SIMT kernels (tile heights 64 / 128) are made here so
    // that a prepared evaluation allocates nothing
    if (family_of(precision) == 0) {
        ensure_stores<double>(H, 0);
        ensure_workspace<double>(H, 0, r_max);
        for (Launch& l : H.dev->launches) tiles_for(l, 64);
    } else if (precision == GOFMM_PREC_FP32) {
        ensure_stores<float>(H, 1);
        ensure_workspace<float>(H, 1, r_max);
        for (Launch& l : H.dev->launches) tiles_for(l, 128);
    } else {
        // the tensor-core tiles are built from the FP32 stores once
        if (!tc_ready(*H.dev, 1, precision)) ensure_stores<float>(H, 1);
        tc_prepare(H, *H.dev, r_max, precision);
    }
    CUDA_OK(cudaDeviceSynchronize());
}

template <typename T, int TM, int TN>
static int run_simt(Handle& H, const T* W, int64_t ldw, T* U, int64_t ldu, int r, cudaStream_t s) {
    DeviceState& D = *H.dev;
    Family& F = D.fam[std::is_same<T, double>::value ? 0 : 1];
    constexpr int BM = 16 * TM, BN = 16 * TN;
    T* WT = static_cast<T*>(F.WT);
    T* WTIL = static_cast<T*>(F.WTIL);
    T* UTIL = static_cast<T*>(F.UTIL);
    int launches = 0;
    const bool timing = H.timing != 0 && D.ev_ok;
    D.last_fused = false;
    if (timing) CUDA_OK(cudaEventRecord(D.ev[0], s));
    {
        dim3 blk(32, 8), grid(unsigned((D.n + 7) / 8));
        gather_rows_kernel<T><<<grid, blk, 0, s>>>(W, ldw, D.d_idx, WT, D.n, r);
        CUDA_OK(cudaGetLastError());
        ++launches;
    }
    if (timing) CUDA_OK(cudaEventRecord(D.ev[1], s));
    GemmParams<T> p{};
    p.kstore = static_cast<const T*>(F.kstore);
    p.pstore = static_cast<const T*>(F.pstore);
    p.b0 = WT; p.b1 = WTIL; p.b2 = UTIL;
    p.ldb = r;
    p.idx = D.d_idx;
    p.pts = std::is_same<T, double>::value ? reinterpret_cast<const T*>(D.d_pts64)
                                           : reinterpret_cast<const T*>(D.d_pts32);
    p.dim = H.K.dim;
    p.gen_kind = H.K.kind;
    p.gen_inv = H.K.kind == GOFMM_GEN_GAUSSIAN ? T(1.0 / (2.0 * H.K.h * H.K.h)) : T(1.0 / (H.K.h * H.K.h));
    p.gen_shift = T(H.K.shift);
    p.r = r;
    p.out_wtil = WTIL;
    p.out_util = UTIL;
    p.out_u = U;
    p.ldu = ldu;
    p.perm = D.d_idx;
    int stage_done = 1;  // events ev[0..stage_done] recorded; ev[i+1] closes stage i
    for (size_t li = 0; li < D.launches.size(); ++li) {
        Launch& l = D.launches[li];
        while (timing && stage_done < l.stage) { CUDA_OK(cudaEventRecord(D.ev[++stage_done], s)); }
        auto tl = tiles_for(l, BM);
        if (tl.second == 0) continue;
        p.tasks = l.d_tasks;
        p.slabs = l.d_slabs;
        p.tiles = tl.first;
        dim3 grid(unsigned(tl.second), unsigned((r + BN - 1) / BN));
        gemm_simt_kernel<T, TM, TN><<<grid, 256, 0, s>>>(p);
        CUDA_OK(cudaGetLastError());
        ++launches;
    }
    while (timing && stage_done < 5) { CUDA_OK(cudaEventRecord(D.ev[++stage_done], s)); }
    return launches;
}

// The SIMT launch sequence of run_simt with the three scratch buffers given
// by the caller; it takes no timing events and creates no tile lists, so it
// never allocates (the handle must have been prepared for the precision).
template <typename T, int TM, int TN>
static int run_simt_on(Handle& H, const T* W, int64_t ldw, T* U, int64_t ldu, int r, cudaStream_t s, T* WT,
                       T* WTIL, T* UTIL) {
    DeviceState& D = *H.dev;
    Family& F = D.fam[std::is_same<T, double>::value ? 0 : 1];
    constexpr int BM = 16 * TM, BN = 16 * TN;
    for (Launch& l : D.launches)
        if (l.tiles.find(BM) == l.tiles.end())
            fail(GOFMM_ERR_ARG, "handle not prepared for this precision: call gofmm_prepare first");
    int launches = 0;
    {
        dim3 blk(32, 8), grid(unsigned((D.n + 7) / 8));
        gather_rows_kernel<T><<<grid, blk, 0, s>>>(W, ldw, D.d_idx, WT, D.n, r);
        CUDA_OK(cudaGetLastError());
        ++launches;
    }
    GemmParams<T> p{};
    p.kstore = static_cast<const T*>(F.kstore);
    p.pstore = static_cast<const T*>(F.pstore);
    p.b0 = WT; p.b1 = WTIL; p.b2 = UTIL;
    p.ldb = r;
    p.idx = D.d_idx;
    p.pts = std::is_same<T, double>::value ? reinterpret_cast<const T*>(D.d_pts64)
                                           : reinterpret_cast<const T*>(D.d_pts32);
    p.dim = H.K.dim;
    p.gen_kind = H.K.kind;
    p.gen_inv = H.K.kind == GOFMM_GEN_GAUSSIAN ? T(1.0 / (2.0 * H.K.h * H.K.h)) : T(1.0 / (H.K.h * H.K.h));
    p.gen_shift = T(H.K.shift);
    p.r = r;
    p.out_wtil = WTIL;
    p.out_util = UTIL;
    p.out_u = U;
    p.ldu = ldu;
    p.perm = D.d_idx;
    for (Launch& l : D.launches) {
        const auto tl = l.tiles.at(BM);
        if (tl.second == 0) continue;
        p.tasks = l.d_tasks;
        p.slabs = l.d_slabs;
        p.tiles = tl.first;
        dim3 grid(unsigned(tl.second), unsigned((r + BN - 1) / BN));
        gemm_simt_kernel<T, TM, TN><<<grid, 256, 0, s>>>(p);
        CUDA_OK(cudaGetLastError());
        ++launches;
    }
    return launches;
}

int simt_evaluate_on(Handle& H, const void* W, int64_t ldw, void* U, int64_t ldu, int r, int precision,
                     cudaStream_t s, void* WT, void* WTIL, void* UTIL) {
    if (precision == GOFMM_PREC_FP64)
        return run_simt_on<double, 4, 4>(H, static_cast<const double*>(W), ldw, static_cast<double*>(U), ldu, r,
                                         s, static_cast<double*>(WT), static_cast<double*>(WTIL),
                                         static_cast<double*>(UTIL));
    return run_simt_on<float, 8, 8>(H, static_cast<const float*>(W), ldw, static_cast<float*>(U), ldu, r, s,
                                    static_cast<float*>(WT), static_cast<float*>(WTIL), static_cast<float*>(UTIL));
}

void device_evaluate(Handle& H, const void* W, int64_t ldw, void* U, int64_t ldu, int64_t r, int dtype,
                     int precision, void* stream, int host_buffers) {
    if (!W || !U) fail(GOFMM_ERR_ARG, "W and U must not be NULL");
    if (r < 1 || r > (int64_t(1) << 30)) fail(GOFMM_ERR_ARG, "r must be >= 1");
    if (ldw < r || ldu < r) fail(GOFMM_ERR_ARG, "leading dimensions must be >= r");
    if (precision < GOFMM_PREC_FP64 || precision > GOFMM_PREC_BF16X3) fail(GOFMM_ERR_ARG, "unknown precision");
    if (dtype != GOFMM_DTYPE_F64 && dtype != GOFMM_DTYPE_F32) fail(GOFMM_ERR_ARG, "unknown dtype");
    if ((precision == GOFMM_PREC_FP64) != (dtype == GOFMM_DTYPE_F64))
        fail(GOFMM_ERR_UNSUPPORTED, "FP64 precision needs F64 data and the other precisions F32 data");
    const size_t es = dtype == GOFMM_DTYPE_F64 ? 8 : 4;
    {
        const char* w0 = static_cast<const char*>(W);
        const char* u0 = static_cast<const char*>(U);
        const size_t span_w = size_t(H.st.n - 1) * size_t(ldw) * es + size_t(r) * es;
        const size_t span_u = size_t(H.st.n - 1) * size_t(ldu) * es + size_t(r) * es;
        if (w0 < u0 + span_u && u0 < w0 + span_w) fail(GOFMM_ERR_ARG, "W and U overlap");
    }
    DeviceGuard g(H.st.prm.device);
    const int fi = family_of(precision);
    Family* F = H.dev ? &H.dev->fam[fi] : nullptr;
    const bool ready = precision <= GOFMM_PREC_FP32 ? (H.dev && F->stores && F->ws_r >= r)
                                                    : (H.dev && tc_ready(*H.dev, r, precision));
    if (!ready) device_prepare(H, std::max<int64_t>(r, F ? F->ws_r : 0), precision);
    DeviceState& D = *H.dev;
    F = &D.fam[fi];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const void* Wd = W;
    void* Ud = U;
    int64_t ldw_d = ldw, ldu_d = ldu;
    const bool async = host_buffers == 2;
    // synchronous calls overlap their own column halves with the copies;
    // asynchronous calls overlap whole calls (the copies of one with the
    // evaluation of the next), so they run as one chunk on the copy streams
    const bool pipelined = host_buffers && H.timing == 0 && (async || r >= 2 * kHostChunk);
    const int64_t chunk = async ? r : host_chunk(r);
    int slot = 0;  // staging slot of this call
    if (host_buffers) {
        if (fi == 0) ensure_staging<double>(H, 0, r, async);
        else ensure_staging<float>(H, 1, r, async);
        F = &D.fam[fi];
        if (async) {  // asynchronous calls take the slots in turn
            slot = F->stage_next;
            F->stage_next = (F->stage_next + 1) % Family::kStageSlots;
        }
        // the slot's previous call must have copied its U out first
        CUDA_OK(cudaStreamWaitEvent(s, F->slot_free[slot], 0));
        if (!pipelined)
            CUDA_OK(cudaMemcpy2DAsync(F->sW[slot], size_t(r) * es, W, size_t(ldw) * es, size_t(r) * es,
                                      size_t(D.n), cudaMemcpyHostToDevice, s));
        Wd = F->sW[slot];
        Ud = F->sU[slot];
        ldw_d = ldu_d = r;
    }
    auto launch_all = [&](cudaStream_t st) -> int {
        if (precision == GOFMM_PREC_FP64)
            return run_simt<double, 4, 4>(H, static_cast<const double*>(Wd), ldw_d, static_cast<double*>(Ud),
                                          ldu_d, int(r), st);
        if (precision == GOFMM_PREC_FP32)
            return run_simt<float, 8, 8>(H, static_cast<const float*>(Wd), ldw_d, static_cast<float*>(Ud), ldu_d,
                                         int(r), st);
        return tc_run(H, D, static_cast<const float*>(Wd), ldw_d, static_cast<float*>(Ud), ldu_d, int(r),
                      precision, st);
    };
    if (pipelined) {
        // Host buffers: the columns of W and U are independent, so the
        // evaluation runs over column chunks while chunk k + 1 is copied in
        // and chunk k - 1 copied out on two copy streams.
        F = &D.fam[fi];
        if (!D.h2d_stream) {
            CUDA_OK(cudaStreamCreateWithFlags(&D.h2d_stream, cudaStreamNonBlocking));
            CUDA_OK(cudaStreamCreateWithFlags(&D.d2h_stream, cudaStreamNonBlocking));
        }
        const int64_t nch = (r + chunk - 1) / chunk;
        while (int64_t(D.pipe_events.size()) < 2 * nch + 1) {
            cudaEvent_t e = nullptr;
            CUDA_OK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            D.pipe_events.push_back(e);
        }
        if (async) {
            // the copies in wait only for the slot to be free, so that they
            // overlap the evaluation of the call before (W is read as it is
            // when the call is made)
            CUDA_OK(cudaStreamWaitEvent(D.h2d_stream, F->slot_free[slot], 0));
        } else {
            cudaEvent_t start = D.pipe_events[2 * size_t(nch)];
            CUDA_OK(cudaEventRecord(start, s));  // the copies follow the caller's earlier work
            CUDA_OK(cudaStreamWaitEvent(D.h2d_stream, start, 0));
        }
        char* dW = static_cast<char*>(F->sW[slot]);
        char* dU = static_cast<char*>(F->sU[slot]);
        for (int64_t k = 0; k < nch; ++k) {
            const int64_t c0 = k * chunk, ck = std::min<int64_t>(chunk, r - c0);
            CUDA_OK(cudaMemcpy2DAsync(dW + size_t(c0) * es, size_t(r) * es, static_cast<const char*>(W) + size_t(c0) * es,
                                      size_t(ldw) * es, size_t(ck) * es, size_t(D.n), cudaMemcpyHostToDevice,
                                      D.h2d_stream));
            CUDA_OK(cudaEventRecord(D.pipe_events[2 * size_t(k)], D.h2d_stream));
        }
        int launches = 0;
        for (int64_t k = 0; k < nch; ++k) {
            const int64_t c0 = k * chunk, ck = std::min<int64_t>(chunk, r - c0);
            CUDA_OK(cudaStreamWaitEvent(s, D.pipe_events[2 * size_t(k)], 0));
            Wd = dW + size_t(c0) * es;
            Ud = dU + size_t(c0) * es;
            if (precision == GOFMM_PREC_FP64)
                launches += run_simt<double, 4, 4>(H, static_cast<const double*>(Wd), r, static_cast<double*>(Ud), r,
                                                   int(ck), s);
            else if (precision == GOFMM_PREC_FP32)
                launches += run_simt<float, 8, 8>(H, static_cast<const float*>(Wd), r, static_cast<float*>(Ud), r,
                                                  int(ck), s);
            else
                launches += tc_run(H, D, static_cast<const float*>(Wd), r, static_cast<float*>(Ud), r, int(ck),
                                   precision, s);
            CUDA_OK(cudaEventRecord(D.pipe_events[2 * size_t(k) + 1], s));
            CUDA_OK(cudaStreamWaitEvent(D.d2h_stream, D.pipe_events[2 * size_t(k) + 1], 0));
            CUDA_OK(cudaMemcpy2DAsync(static_cast<char*>(U) + size_t(c0) * es, size_t(ldu) * es, dU + size_t(c0) * es,
                                      size_t(r) * es, size_t(ck) * es, size_t(D.n), cudaMemcpyDeviceToHost,
                                      D.d2h_stream));
        }
        D.last_launches = launches;
        CUDA_OK(cudaEventRecord(F->slot_free[slot], D.d2h_stream));
        if (!async) {
            CUDA_OK(cudaStreamSynchronize(D.d2h_stream));
            CUDA_OK(cudaStreamSynchronize(s));
        }
        return;
    }
    if (H.timing != 0 || host_buffers) {
        D.last_launches = launch_all(s);
    } else {
        // replay the launch sequence as a CUDA graph once the same call repeats
        if (precision > GOFMM_PREC_FP32 && tc_error(D))
            fail(GOFMM_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait (code " +
                                        std::to_string(tc_error(D)) + ")");
        auto& e = D.graphs[std::make_tuple(precision, r, Wd, ldw_d, Ud, ldu_d)];
        ++e.calls;
        if (!e.exec && e.calls >= 2) {
            cudaGraph_t gr = nullptr;
            CUDA_OK(cudaStreamBeginCapture(D.capture_stream, cudaStreamCaptureModeThreadLocal));
            int n = 0;
            try {
                n = launch_all(D.capture_stream);
            } catch (...) {
                cudaStreamEndCapture(D.capture_stream, &gr);
                if (gr) cudaGraphDestroy(gr);
                throw;
            }
            CUDA_OK(cudaStreamEndCapture(D.capture_stream, &gr));
            const cudaError_t ie = cudaGraphInstantiate(&e.exec, gr, 0);
            cudaGraphDestroy(gr);
            CUDA_OK(ie);
            e.launches = n;
        }
        if (e.exec) {
            CUDA_OK(cudaGraphLaunch(e.exec, s));
            D.last_launches = e.launches;
        } else {
            D.last_launches = launch_all(s);
        }
    }
    if (host_buffers) {
        CUDA_OK(cudaMemcpy2DAsync(U, size_t(ldu) * es, Ud, size_t(r) * es, size_t(r) * es, size_t(D.n),
                                  cudaMemcpyDeviceToHost, s));
        CUDA_OK(cudaEventRecord(F->slot_free[slot], s));
        if (!async) CUDA_OK(cudaStreamSynchronize(s));
    }
}

void device_trim(Handle& H) {
    if (!H.dev) return;
    DeviceGuard g(H.st.prm.device);
    CUDA_OK(cudaDeviceSynchronize());
    clear_graphs(*H.dev);
    for (Family& F : H.dev->fam) {
        dfree(F.kstore);
        dfree(F.pstore);
        dfree(F.WT);
        dfree(F.WTIL);
        dfree(F.UTIL);
        for (int k = 0; k < Family::kStageSlots; ++k) {
            dfree(F.sW[k]);
            dfree(F.sU[k]);
        }
        for (cudaEvent_t e : F.slot_free)
            if (e) cudaEventDestroy(e);
        F = Family{};
    }
}

void device_synchronize(Handle& H, void* stream) {
    if (!H.dev) return;
    DeviceGuard g(H.st.prm.device);
    CUDA_OK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    if (H.dev->d2h_stream) CUDA_OK(cudaStreamSynchronize(H.dev->d2h_stream));  // asynchronous host-buffer calls
    CUDA_OK(cudaGetLastError());
    if (const int e = tc_error(*H.dev)) {
        tc_clear_error(*H.dev);  // reported once; the handle stays usable
        fail(GOFMM_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait (code " + std::to_string(e) + ")");
    }
}

void device_set_tc_config(Handle& H, int precision, int piece, int schedule, int order) {
    if (precision != GOFMM_PREC_TF32 && precision != GOFMM_PREC_BF16 && precision != GOFMM_PREC_BF16X3)
        fail(GOFMM_ERR_ARG, "the launch configuration belongs to a tensor-core precision (TF32, BF16, BF16X3)");
    if (piece != 128 && piece != 256) fail(GOFMM_ERR_ARG, "piece must be 128 or 256");
    if (schedule < GOFMM_SCHED_FUSED || schedule > GOFMM_SCHED_HYBRID) fail(GOFMM_ERR_ARG, "unknown schedule");
    if (order != GOFMM_ORDER_CRITICAL && order != GOFMM_ORDER_LOCAL && order != GOFMM_ORDER_SCHEDULE &&
        order != GOFMM_ORDER_READY && order != GOFMM_ORDER_LEVELS)
        fail(GOFMM_ERR_ARG, "unknown order");
    const int mode = mode_of(precision);
    if (piece != H.tc_piece[mode] && H.inflight > 0)
        fail(GOFMM_ERR_ARG, "a serving engine holds requests of this handle: drain it before changing the plan");
    const bool replan = piece != H.tc_piece[mode] && H.dev && H.dev->tc && H.dev->tc->prec[mode];
    H.tc_schedule[mode] = schedule;
    H.tc_order[mode] = order;
    if (!H.dev) {
        H.tc_piece[mode] = piece;
        return;
    }
    DeviceGuard g(H.st.prm.device);
    clear_graphs(*H.dev);  // captured launches carry the old configuration
    if (!replan) {
        H.tc_piece[mode] = piece;
        if (H.dev->tc && H.dev->tc->prec[mode]) {
            // tile lists of the order now selected
            const int64_t r_cap = H.dev->tc->prec[mode]->r_cap;
            if (r_cap > 0) tc_prepare(H, *H.dev, r_cap, precision);
        }
        return;
    }
    const int64_t r_cap = H.dev->tc->prec[mode]->r_cap;
    tc_drop_plan(*H.dev, precision);
    H.tc_piece[mode] = piece;
    ++H.plan_epoch;
    device_prepare(H, std::max<int64_t>(r_cap, 1), precision);
}

void device_stall_next(Handle& H, int precision) {
    if (!H.dev) fail(GOFMM_ERR_ARG, "handle not prepared: call gofmm_prepare first");
    DeviceGuard g(H.st.prm.device);
    tc_stall_next(*H.dev, precision);
    clear_graphs(*H.dev);  // the next call launches directly
}

void device_stage_times(Handle& H, float* ms, int n) {
    if (!H.dev || !H.dev->ev_ok) fail(GOFMM_ERR_ARG, "no evaluation recorded");
    DeviceState& D = *H.dev;
    DeviceGuard g(H.st.prm.device);
    CUDA_OK(cudaEventSynchronize(D.ev[5]));
    float t[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 5; ++i) CUDA_OK(cudaEventElapsedTime(&t[i], D.ev[i], D.ev[i + 1]));
    CUDA_OK(cudaEventElapsedTime(&t[5], D.ev[0], D.ev[5]));
    if (D.last_fused) {  // gather, then one launch for every grouped GEMM
        t[1] = t[1] + t[2] + t[3] + t[4];
        t[2] = t[3] = t[4] = 0.f;
    }
    for (int i = 0; i < n && i < 6; ++i) ms[i] = t[i];
    if (n > 6) ms[6] = float(D.last_launches);
}

void device_destroy(Handle& H) {
    if (!H.dev) return;
    DeviceState* D = H.dev;
    H.dev = nullptr;
    int old = -1;
    cudaGetDevice(&old);
    cudaSetDevice(D->device);
    cudaDeviceSynchronize();
    clear_graphs(*D);
    if (D->capture_stream) cudaStreamDestroy(D->capture_stream);
    if (D->h2d_stream) cudaStreamDestroy(D->h2d_stream);
    if (D->d2h_stream) cudaStreamDestroy(D->d2h_stream);
    for (cudaEvent_t e : D->pipe_events) cudaEventDestroy(e);
    tc_destroy(*D);
    for (Launch& l : D->launches) {
        dfree(l.d_tasks);
        dfree(l.d_slabs);
        for (auto& kv : l.tiles) dfree(kv.second.first);
    }
    dfree(D->d_idx); dfree(D->d_pts64); dfree(D->d_pts32); dfree(D->d_kblocks);
    for (Family& F : D->fam) {
        dfree(F.kstore); dfree(F.pstore); dfree(F.WT); dfree(F.WTIL); dfree(F.UTIL);
        for (int k = 0; k < Family::kStageSlots; ++k) {
            dfree(F.sW[k]);
            dfree(F.sU[k]);
        }
        for (cudaEvent_t e : F.slot_free)
            if (e) cudaEventDestroy(e);
    }
    if (D->ev_ok)
        for (auto& e : D->ev) cudaEventDestroy(e);
    delete D;
    if (old >= 0) cudaSetDevice(old);
}

}  // namespace gofmm
