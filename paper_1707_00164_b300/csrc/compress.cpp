// Host-side GOFMM compression in FP64 (Alg. 2 of the paper): neighbour
// search, metric ball tree (Alg. 1), near lists (Alg. 3 with the budget
// ballot), far lists (Algs. 4-5, or the symmetric same-level reading), and
// skeletons with interpolation matrices by adaptive ID (Alg. 6, pivoted QR +
// triangular solve).  Parallel over tree nodes / rows with OpenMP; every
// result is independent of the thread count.
#include <omp.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>

#include "gofmm_internal.hpp"

namespace gofmm {

void fail(int code, const std::string& msg) { throw Error{code, msg}; }

void partial_shuffle(std::vector<int64_t>& a, int64_t k, uint64_t key) {
    const int64_t n = int64_t(a.size());
    k = std::min(k, n);
    for (int64_t t = 0; t < k; ++t) {
        const uint64_t u = sm_output(key, uint64_t(t));
        const int64_t j = t + int64_t(u % uint64_t(n - t));
        std::swap(a[t], a[j]);
    }
}

// ----------------------------------------------------------------- entries --
void Entries::block(const int64_t* I, int64_t nI, const int64_t* J, int64_t nJ,
                    double* out) const {
    if (nI == 0 || nJ == 0) return;
    if (kind == GOFMM_GEN_CALLBACK) {
        const int rc = fn(ctx, I, nI, J, nJ, out);
        if (rc != 0) fail(GOFMM_ERR_CALLBACK, "entry callback returned " + std::to_string(rc));
        for (int64_t t = 0; t < nI * nJ; ++t)
            if (!std::isfinite(out[t])) fail(GOFMM_ERR_NONFINITE, "entry callback produced a non-finite entry");
        return;
    }
    const double two_h2 = 2.0 * h * h;
    const double h2 = h * h;
    for (int64_t i = 0; i < nI; ++i) {
        const double* xi = &pts[size_t(I[i]) * dim];
        for (int64_t j = 0; j < nJ; ++j) {
            const double* xj = &pts[size_t(J[j]) * dim];
            double acc = 0.0;
            for (int k = 0; k < dim; ++k) {
                const double d = xi[k] - xj[k];
                acc += d * d;
            }
            double v = (kind == GOFMM_GEN_GAUSSIAN) ? std::exp(-(acc / two_h2))
                                                    : 1.0 / std::sqrt(1.0 + acc / h2);
            if (I[i] == J[j]) v += shift;
            out[i * nJ + j] = v;
        }
    }
}

double Entries::diag(int64_t i) const {
    double v;
    block(&i, 1, &i, 1, &v);
    return v;
}

int tree_depth(int64_t n, int64_t m) {
    int L = 0;
    while ((n + (int64_t(1) << L) - 1) / (int64_t(1) << L) > m) ++L;
    return L;
}

// Run f(i) for i in [0, n); the first Error thrown by any iteration is
// rethrown after the loop.
template <class F>
static void parallel_for(int64_t n, bool par, F&& f) {
    std::atomic<bool> failed{false};
    Error err{0, ""};
#pragma omp parallel for schedule(dynamic, 1) if (par)
    for (int64_t i = 0; i < n; ++i) {
        if (failed.load(std::memory_order_relaxed)) continue;
        try {
            f(i);
        } catch (const Error& e) {
#pragma omp critical(gofmm_err)
            {
                if (!failed.load()) { err = e; failed.store(true); }
            }
        } catch (const std::bad_alloc&) {
#pragma omp critical(gofmm_err)
            {
                if (!failed.load()) { err = Error{GOFMM_ERR_NOMEM, "host allocation failed"}; failed.store(true); }
            }
        }
    }
    if (failed.load()) throw err;
}

// ------------------------------------------------------------- distances --
// §2.1: Gram-l2 distance (clamped before the square root) and Gram angle.
static inline double dist_value(int kind, double kii, double kjj, double kij) {
    if (kind == GOFMM_DIST_ANGLE) return 1.0 - (kij * kij) / (kii * kjj);
    const double d2 = (kii + kjj) - 2.0 * kij;
    return std::sqrt(std::max(d2, 0.0));
}
// neighbour ranking key: clamped d^2 (Gram-l2) or d (angle)
static inline double knn_key(int kind, double kii, double kjj, double kij) {
    if (kind == GOFMM_DIST_ANGLE) return 1.0 - (kij * kij) / (kii * kjj);
    return std::max((kii + kjj) - 2.0 * kij, 0.0);
}
static inline int metric_of(int distance) {
    return distance == GOFMM_DIST_ANGLE ? GOFMM_DIST_ANGLE : GOFMM_DIST_GRAM_L2;
}

struct Ctx {
    const Entries& K;
    const Params& prm;
    std::vector<double> diagK;
    bool par;
};

// medianSplit of Alg. 1: order by (v, index); the left child takes ceil(n/2).
static void median_split(const std::vector<int64_t>& idx, const std::vector<double>& v,
                         std::vector<int64_t>& lc, std::vector<int64_t>& rc) {
    const size_t n = idx.size();
    std::vector<size_t> o(n);
    std::iota(o.begin(), o.end(), 0);
    std::sort(o.begin(), o.end(), [&](size_t a, size_t b) {
        return v[a] < v[b] || (v[a] == v[b] && idx[a] < idx[b]);
    });
    const size_t half = (n + 1) / 2;
    lc.resize(half);
    rc.resize(n - half);
    for (size_t t = 0; t < half; ++t) lc[t] = idx[o[t]];
    for (size_t t = half; t < n; ++t) rc[t - half] = idx[o[t]];
    std::sort(lc.begin(), lc.end());
    std::sort(rc.begin(), rc.end());
}

static std::vector<double> dist_to(const Ctx& c, const std::vector<int64_t>& idx, int64_t p, int kind) {
    const size_t n = idx.size();
    std::vector<double> col(n), d(n);
    c.K.block(idx.data(), int64_t(n), &p, 1, col.data());
    for (size_t i = 0; i < n; ++i) d[i] = dist_value(kind, c.diagK[idx[i]], c.diagK[p], col[i]);
    return d;
}

static size_t first_argmax(const std::vector<double>& v) {
    size_t b = 0;
    for (size_t i = 1; i < v.size(); ++i)
        if (v[i] > v[b]) b = i;
    return b;
}

// Alg. 1 (metricSplit) with the sampled centroid of §2.1.
static void metric_split(const Ctx& c, const std::vector<int64_t>& idx, int64_t h,
                         std::vector<int64_t>& lc, std::vector<int64_t>& rc) {
    const int kind = metric_of(c.prm.distance);
    const int64_t n = int64_t(idx.size());
    const int64_t nc = std::min<int64_t>(c.prm.n_centroid, n);
    std::vector<int64_t> C = idx;
    partial_shuffle(C, nc, stream_key(c.prm.seed, kCentroid, uint64_t(h)));
    C.resize(nc);
    std::vector<double> Kc(size_t(n * nc));
    c.K.block(idx.data(), n, C.data(), nc, Kc.data());
    std::vector<double> S(n, 0.0), score(n);
    for (int64_t t = 0; t < nc; ++t)
        for (int64_t i = 0; i < n; ++i) S[i] = S[i] + Kc[i * nc + t];
    if (kind == GOFMM_DIST_GRAM_L2) {
        for (int64_t i = 0; i < n; ++i) score[i] = c.diagK[idx[i]] - 2.0 * S[i] / double(nc);
    } else {
        std::vector<double> Kcc(size_t(nc * nc));
        c.K.block(C.data(), nc, C.data(), nc, Kcc.data());
        double acc = 0.0;
        for (int64_t t = 0; t < nc * nc; ++t) acc += Kcc[t];
        const double cc = acc / double(nc * nc);
        for (int64_t i = 0; i < n; ++i) {
            const double a = S[i] / double(nc);
            score[i] = 1.0 - (a * a) / (c.diagK[idx[i]] * cc);
        }
    }
    const int64_t p = idx[first_argmax(score)];
    std::vector<double> dp = dist_to(c, idx, p, kind);
    const int64_t q = idx[first_argmax(dp)];
    std::vector<double> dq = dist_to(c, idx, q, kind);
    std::vector<double> v(n);
    for (int64_t i = 0; i < n; ++i) v[i] = dp[i] - dq[i];
    median_split(idx, v, lc, rc);
}

// Random projection split of the neighbour search: p, q drawn at random.
static void random_split(const Ctx& c, const std::vector<int64_t>& idx, uint64_t key,
                         std::vector<int64_t>& lc, std::vector<int64_t>& rc) {
    const int kind = metric_of(c.prm.distance);
    const uint64_t n = idx.size();
    const int64_t p = idx[sm_output(key, 0) % n];
    int64_t q = p;
    for (uint64_t t = 1; q == p; ++t) q = idx[sm_output(key, t) % n];
    std::vector<double> dp = dist_to(c, idx, p, kind), dq = dist_to(c, idx, q, kind);
    std::vector<double> v(n);
    for (size_t i = 0; i < n; ++i) v[i] = dp[i] - dq[i];
    median_split(idx, v, lc, rc);
}

// PRE-order SPLI over a complete tree of depth tree_depth(n, m).
// mode: 0 metric (or lexicographic/random per prm.distance), 1 random
// projection for ANN iteration `it`.
static std::vector<std::vector<int64_t>> build_tree(const Ctx& c, int mode, int it) {
    const int64_t n = c.K.n;
    const int L = tree_depth(n, c.prm.m);
    std::vector<std::vector<int64_t>> nodes(size_t((int64_t(2) << L) - 1));
    nodes[0].resize(n);
    std::iota(nodes[0].begin(), nodes[0].end(), 0);
    std::vector<int64_t> rank;
    if (mode == 0 && c.prm.distance == GOFMM_DIST_RANDOM) {
        std::vector<int64_t> a(n);
        std::iota(a.begin(), a.end(), 0);
        partial_shuffle(a, n, stream_key(c.prm.seed, kRandomPerm, 0));
        rank.resize(n);
        for (int64_t t = 0; t < n; ++t) rank[a[t]] = t;
    }
    for (int lvl = 0; lvl < L; ++lvl) {
        const int64_t first = (int64_t(1) << lvl) - 1, cnt = int64_t(1) << lvl;
        parallel_for(cnt, c.par, [&](int64_t t) {
            const int64_t h = first + t;
            const std::vector<int64_t>& idx = nodes[h];
            std::vector<int64_t>& lc = nodes[2 * h + 1];
            std::vector<int64_t>& rc = nodes[2 * h + 2];
            if (mode == 1) {
                random_split(c, idx, stream_key(c.prm.seed, kAnnSplit, (uint64_t(it) << 24) | uint64_t(h)), lc, rc);
            } else if (c.prm.distance == GOFMM_DIST_LEXICOGRAPHIC) {
                const size_t half = (idx.size() + 1) / 2;
                lc.assign(idx.begin(), idx.begin() + half);
                rc.assign(idx.begin() + half, idx.end());
            } else if (c.prm.distance == GOFMM_DIST_RANDOM) {
                std::vector<double> v(idx.size());
                for (size_t i = 0; i < idx.size(); ++i) v[i] = double(rank[idx[i]]);
                median_split(idx, v, lc, rc);
            } else {
                metric_split(c, idx, h, lc, rc);
            }
        });
    }
    return nodes;
}

// ------------------------------------------------------------------ kNN --
using Cand = std::pair<double, int64_t>;  // (key, index), ordered lexicographically

// Exhaustive kappa nearest neighbours of `rows` (an index is its own nearest).
static void knn_exact(const Ctx& c, const std::vector<int64_t>& rows, int kappa,
                      std::vector<int64_t>& out_c, std::vector<double>& out_k) {
    const int64_t n = c.K.n;
    const int kind = metric_of(c.prm.distance);
    const int64_t R = int64_t(rows.size());
    out_c.assign(size_t(R * kappa), -1);
    out_k.assign(size_t(R * kappa), INFINITY);
    std::vector<int64_t> allj(n);
    std::iota(allj.begin(), allj.end(), 0);
    const int64_t B = 32;
    parallel_for((R + B - 1) / B, c.par, [&](int64_t blk) {
        const int64_t r0 = blk * B, nb = std::min(B, R - r0);
        std::vector<double> Kb(size_t(nb * n));
        c.K.block(&rows[r0], nb, allj.data(), n, Kb.data());
        std::vector<Cand> cand(n);
        for (int64_t t = 0; t < nb; ++t) {
            const int64_t i = rows[r0 + t];
            for (int64_t j = 0; j < n; ++j) cand[j] = Cand(knn_key(kind, c.diagK[i], c.diagK[j], Kb[t * n + j]), j);
            std::nth_element(cand.begin(), cand.begin() + (kappa - 1), cand.end());
            std::sort(cand.begin(), cand.begin() + kappa);
            for (int k = 0; k < kappa; ++k) {
                out_c[(r0 + t) * kappa + k] = cand[k].second;
                out_k[(r0 + t) * kappa + k] = cand[k].first;
            }
        }
    });
}

// Neighbour search of Alg. 2 steps 1-3: exhaustive for small N, otherwise
// random projection trees with exhaustive leaf search, until the recall on
// 100 sampled indices reaches the target or the iteration limit.
static std::vector<int64_t> all_nearest_neighbors(const Ctx& c, int& iters, double& recall) {
    const int64_t n = c.K.n;
    const int kappa = int(std::min<int64_t>(c.prm.kappa, n));
    std::vector<int64_t> cur_c;
    std::vector<double> cur_k;
    if (n <= c.prm.knn_exact_max) {
        std::vector<int64_t> rows(n);
        std::iota(rows.begin(), rows.end(), 0);
        knn_exact(c, rows, kappa, cur_c, cur_k);
        iters = 0;
        recall = 1.0;
        return cur_c;
    }
    cur_c.assign(size_t(n * kappa), -1);
    cur_k.assign(size_t(n * kappa), INFINITY);
    std::vector<int64_t> sample(n);
    std::iota(sample.begin(), sample.end(), 0);
    const int64_t ns = std::min<int64_t>(100, n);
    partial_shuffle(sample, ns, stream_key(c.prm.seed, kAnnRecall, 0));
    sample.resize(ns);
    std::sort(sample.begin(), sample.end());
    std::vector<int64_t> ex_c;
    std::vector<double> ex_k;
    knn_exact(c, sample, kappa, ex_c, ex_k);
    const int kind = metric_of(c.prm.distance);
    recall = 0.0;
    iters = 0;
    for (int it = 1; it <= c.prm.ann_max_iter; ++it) {
        iters = it;
        auto nodes = build_tree(c, 1, it);
        const int L = tree_depth(n, c.prm.m);
        const int64_t first_leaf = (int64_t(1) << L) - 1, nl = int64_t(1) << L;
        parallel_for(nl, c.par, [&](int64_t b) {
            const std::vector<int64_t>& lf = nodes[first_leaf + b];
            const int64_t ls = int64_t(lf.size());
            std::vector<double> Kb(size_t(ls * ls));
            c.K.block(lf.data(), ls, lf.data(), ls, Kb.data());
            std::vector<Cand> cand;
            cand.reserve(size_t(kappa + ls));
            for (int64_t t = 0; t < ls; ++t) {
                const int64_t i = lf[t];
                cand.clear();
                for (int k = 0; k < kappa; ++k) {
                    const int64_t j = cur_c[i * kappa + k];
                    // unfilled slots: distinct placeholder ids >= n, infinite key
                    cand.emplace_back(j < 0 ? INFINITY : cur_k[i * kappa + k], j < 0 ? n + k : j);
                }
                for (int64_t u = 0; u < ls; ++u)
                    cand.emplace_back(knn_key(kind, c.diagK[i], c.diagK[lf[u]], Kb[t * ls + u]), lf[u]);
                std::sort(cand.begin(), cand.end());
                int k = 0;
                for (size_t u = 0; u < cand.size() && k < kappa; ++u) {
                    if (u > 0 && cand[u].second == cand[u - 1].second) continue;
                    const bool ph = cand[u].second >= n;
                    cur_c[i * kappa + k] = ph ? -1 : cand[u].second;
                    cur_k[i * kappa + k] = ph ? INFINITY : cand[u].first;
                    ++k;
                }
            }
        });
        int64_t hits = 0;
        for (int64_t t = 0; t < ns; ++t) {
            const int64_t i = sample[t];
            for (int k = 0; k < kappa; ++k) {
                const int64_t j = cur_c[i * kappa + k];
                if (j < 0) continue;
                for (int u = 0; u < kappa; ++u)
                    if (ex_c[t * kappa + u] == j) { ++hits; break; }
            }
        }
        recall = double(hits) / double(ns * kappa);
        if (recall >= c.prm.ann_target_recall) break;
    }
    return cur_c;
}

// ---------------------------------------------------------- near / far --
void fill_node_extents(Structure& st) {
    const int L = st.depth;
    const int64_t nn = st.n_nodes();
    st.node_off.assign(nn, 0);
    // node_size of the leaves is set by the caller; aggregate upwards
    for (int lvl = L - 1; lvl >= 0; --lvl)
        for (int64_t h = (int64_t(1) << lvl) - 1; h < (int64_t(2) << lvl) - 1; ++h)
            st.node_size[h] = st.node_size[2 * h + 1] + st.node_size[2 * h + 2];
    for (int lvl = 0; lvl < L; ++lvl)
        for (int64_t h = (int64_t(1) << lvl) - 1; h < (int64_t(2) << lvl) - 1; ++h) {
            st.node_off[2 * h + 1] = st.node_off[h];
            st.node_off[2 * h + 2] = st.node_off[h] + st.node_size[2 * h + 1];
        }
}

// Alg. 3 (LeafNear) with the ballot and budget of §2.2, then symmetrised.
static void leaf_near(Structure& st, const std::vector<int64_t>& knn, int kappa,
                      const std::vector<int64_t>& leaf_of) {
    const int64_t nl = st.n_leaves();
    const int64_t B = int64_t(std::floor(st.prm.budget * double(st.n) / double(st.prm.m)));
    std::vector<std::vector<int64_t>> chosen(nl);
    for (int64_t b = 0; b < nl; ++b) {
        const int64_t h = st.leaf_node(b);
        std::vector<int64_t> votes(nl, 0);
        for (int64_t t = 0; t < st.node_size[h]; ++t) {
            const int64_t i = st.perm[st.node_off[h] + t];
            for (int k = 0; k < kappa; ++k) {
                const int64_t j = knn[i * kappa + k];
                if (j >= 0) ++votes[leaf_of[j]];
            }
        }
        votes[b] = 0;
        std::vector<int64_t> cand;
        for (int64_t a = 0; a < nl; ++a)
            if (votes[a] > 0) cand.push_back(a);
        std::sort(cand.begin(), cand.end(), [&](int64_t x, int64_t y) {
            return votes[x] > votes[y] || (votes[x] == votes[y] && x < y);
        });
        if (int64_t(cand.size()) > B) cand.resize(size_t(std::max<int64_t>(B, 0)));
        chosen[b] = cand;
    }
    st.near.assign(nl, {});
    std::vector<std::vector<char>> m(nl, std::vector<char>(nl, 0));
    for (int64_t b = 0; b < nl; ++b) {
        m[b][b] = 1;
        for (int64_t a : chosen[b]) { m[b][a] = 1; m[a][b] = 1; }
    }
    for (int64_t b = 0; b < nl; ++b)
        for (int64_t a = 0; a < nl; ++a)
            if (m[b][a]) st.near[b].push_back(a);
}

// Symmetric reading of Algs. 4-5: nodes X != Y on one level are far iff no
// leaf below X is near a leaf below Y while their parents are not far.
static void far_symmetric(Structure& st) {
    const int L = st.depth;
    std::vector<std::vector<char>> nm(L + 1);
    const int64_t nl = st.n_leaves();
    nm[L].assign(size_t(nl * nl), 0);
    for (int64_t b = 0; b < nl; ++b)
        for (int64_t a : st.near[b]) nm[L][b * nl + a] = 1;
    for (int lvl = L - 1; lvl >= 0; --lvl) {
        const int64_t k = int64_t(1) << lvl, k2 = 2 * k;
        nm[lvl].assign(size_t(k * k), 0);
        const auto& c = nm[lvl + 1];
        for (int64_t x = 0; x < k; ++x)
            for (int64_t y = 0; y < k; ++y)
                nm[lvl][x * k + y] = c[(2 * x) * k2 + 2 * y] | c[(2 * x) * k2 + 2 * y + 1] |
                                     c[(2 * x + 1) * k2 + 2 * y] | c[(2 * x + 1) * k2 + 2 * y + 1];
    }
    st.far.assign(st.n_nodes(), {});
    for (int lvl = 1; lvl <= L; ++lvl) {
        const int64_t base = (int64_t(1) << lvl) - 1, cnt = int64_t(1) << lvl, pc = cnt / 2;
        for (int64_t x = 0; x < cnt; ++x)
            for (int64_t y = 0; y < cnt; ++y)
                if (!nm[lvl][x * cnt + y] && nm[lvl - 1][(x / 2) * pc + y / 2])
                    st.far[base + x].push_back(base + y);
    }
}

// Alg. 4 (FindFar from the root for every leaf) and Alg. 5 (MergeFar in
// postorder), literally.
static void far_paper(Structure& st) {
    const int L = st.depth;
    const int64_t nn = st.n_nodes();
    std::vector<std::vector<int64_t>> far(nn);
    auto leaves_under = [&](int64_t h, int64_t& lo, int64_t& hi) {
        int lvl = 0;
        while ((int64_t(2) << lvl) - 1 <= h) ++lvl;
        lo = (h + 1 - (int64_t(1) << lvl)) << (L - lvl);
        hi = lo + (int64_t(1) << (L - lvl));
    };
    for (int64_t b = 0; b < st.n_leaves(); ++b) {
        const std::vector<int64_t>& nb = st.near[b];
        std::vector<int64_t> stack{0};
        while (!stack.empty()) {
            const int64_t h = stack.back();
            stack.pop_back();
            int64_t lo, hi;
            leaves_under(h, lo, hi);
            bool hit = false;
            for (int64_t a : nb)
                if (a >= lo && a < hi) { hit = true; break; }
            if (hit) {
                if (2 * h + 1 < nn) { stack.push_back(2 * h + 2); stack.push_back(2 * h + 1); }
            } else {
                far[st.leaf_node(b)].push_back(h);
            }
        }
        std::sort(far[st.leaf_node(b)].begin(), far[st.leaf_node(b)].end());
    }
    for (int lvl = L - 1; lvl >= 0; --lvl)
        for (int64_t h = (int64_t(1) << lvl) - 1; h < (int64_t(2) << lvl) - 1; ++h) {
            auto& l = far[2 * h + 1];
            auto& r = far[2 * h + 2];
            std::vector<int64_t> both;
            std::set_intersection(l.begin(), l.end(), r.begin(), r.end(), std::back_inserter(both));
            std::vector<int64_t> merged;
            std::set_union(far[h].begin(), far[h].end(), both.begin(), both.end(), std::back_inserter(merged));
            far[h] = merged;
            std::vector<int64_t> l2, r2;
            std::set_difference(l.begin(), l.end(), both.begin(), both.end(), std::back_inserter(l2));
            std::set_difference(r.begin(), r.end(), both.begin(), both.end(), std::back_inserter(r2));
            l = l2;
            r = r2;
        }
    st.far = far;
}

// -------------------------------------------------------- skeletonization --
// y -= c * x (element-wise; the same rounding on every instruction set, no
// contraction into FMA)
__attribute__((target_clones("avx512f", "avx2", "default"))) static void axpy_sub(double* y, const double* x,
                                                                                double c, int64_t n) {
    for (int64_t i = 0; i < n; ++i) y[i] -= x[i] * c;
}

// Dot product with eight independent partial sums (lets the compiler keep
// several vector lanes busy without reassociating a single sum).
__attribute__((target_clones("avx512f", "avx2", "default"))) static double dot8(const double* a, const double* b,
                                                                              int64_t n) {
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t i = 0;
    for (; i + 8 <= n; i += 8)
        for (int u = 0; u < 8; ++u) s[u] += a[i + u] * b[i + u];
    double t = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
    for (; i < n; ++i) t += a[i] * b[i];
    return t;
}

IdResult interpolative_decomposition(std::vector<double>& A, int64_t m, int64_t n,
                                     int64_t max_rank, double tau) {
    IdResult res;
    res.perm.resize(n);
    std::iota(res.perm.begin(), res.perm.end(), 0);
    std::vector<int64_t>& perm = res.perm;
    const int64_t kmax = std::min(std::min(m, n), max_rank);
    std::vector<double> v(m);
    double r00 = 0.0;
    int64_t s = 0;
    for (int64_t k = 0; k < kmax; ++k) {
        // pivot: largest recomputed residual norm, ties to the smallest
        // original column position (Businger-Golub)
        double mx = -1.0;
        int64_t jb = k;
        for (int64_t j = k; j < n; ++j) {
            const double* a = &A[size_t(j * m)] + k;
            const double nrm = std::sqrt(dot8(a, a, m - k));
            if (nrm > mx || (nrm == mx && perm[j] < perm[jb])) { mx = nrm; jb = j; }
        }
        if (jb != k) {
            std::swap_ranges(&A[size_t(k * m)], &A[size_t(k * m)] + m, &A[size_t(jb * m)]);
            std::swap(perm[k], perm[jb]);
        }
        const double rkk = mx;
        if (k == 0) r00 = rkk;
        else if (rkk <= tau * r00) break;
        double* ak = &A[size_t(k * m)];
        const double alpha = ak[k] != 0.0 ? -std::copysign(rkk, ak[k]) : -rkk;
        double vn2 = 0.0;
        for (int64_t i = k; i < m; ++i) v[i] = ak[i];
        v[k] -= alpha;
        for (int64_t i = k; i < m; ++i) vn2 += v[i] * v[i];
        if (vn2 > 0.0) {
            for (int64_t j = k + 1; j < n; ++j) {
                double* aj = &A[size_t(j * m)];
                const double dot = dot8(&v[k], aj + k, m - k);
                const double coef = (2.0 / vn2) * dot;
                axpy_sub(aj + k, &v[k], coef, m - k);
            }
        }
        ak[k] = alpha;
        for (int64_t i = k + 1; i < m; ++i) ak[i] = 0.0;
        s = k + 1;
        if (r00 == 0.0) break;
    }
    s = std::max<int64_t>(s, 1);
    res.s = s;
    // P = [I | R11^{-1} R12] Pi^T (COEF of Table 2), s x n in original order
    res.P.assign(size_t(s * n), 0.0);
    for (int64_t t = 0; t < s; ++t) res.P[size_t(t * n + perm[t])] = 1.0;
    bool nonsingular = true;
    for (int64_t t = 0; t < s; ++t)
        if (A[size_t(t * m + t)] == 0.0) nonsingular = false;
    if (nonsingular) {
        std::vector<double> x(s);
        for (int64_t c = s; c < n; ++c) {
            const double* r12 = &A[size_t(c * m)];
            for (int64_t i = s - 1; i >= 0; --i) {
                double t = r12[i];
                for (int64_t j = i + 1; j < s; ++j) t -= A[size_t(j * m + i)] * x[j];
                x[i] = t / A[size_t(i * m + i)];
            }
            for (int64_t i = 0; i < s; ++i) res.P[size_t(i * n + perm[c])] = x[i];
        }
    }
    return res;
}

// Neighbour-based importance sampling of I' (§2.2): neighbours of the node
// outside it by decreasing count (ties to the smaller index), then uniform
// draws without replacement from the rest of the complement.
static std::vector<int64_t> sample_rows(const Structure& st, const std::vector<int64_t>& knn,
                                        int kappa, int64_t h) {
    const int64_t n = st.n;
    const int64_t sz = st.node_size[h], off = st.node_off[h];
    const int64_t target = st.prm.n_sample > 0 ? st.prm.n_sample : 2 * st.prm.s;
    const int64_t need = std::min(n - sz, target);
    std::vector<char> taken(n, 0);
    for (int64_t t = 0; t < sz; ++t) taken[st.perm[off + t]] = 1;
    std::vector<int32_t> cnt(n, 0);
    std::vector<int64_t> cand;
    for (int64_t t = 0; t < sz; ++t) {
        const int64_t i = st.perm[off + t];
        for (int k = 0; k < kappa; ++k) {
            const int64_t j = knn[i * kappa + k];
            if (j < 0 || taken[j]) continue;
            if (cnt[j]++ == 0) cand.push_back(j);
        }
    }
    std::sort(cand.begin(), cand.end(), [&](int64_t a, int64_t b) {
        return cnt[a] > cnt[b] || (cnt[a] == cnt[b] && a < b);
    });
    if (int64_t(cand.size()) > need) cand.resize(size_t(need));
    if (int64_t(cand.size()) < need) {
        for (int64_t j : cand) taken[j] = 1;
        std::vector<int64_t> rest;
        rest.reserve(size_t(n - sz));
        for (int64_t j = 0; j < n; ++j)
            if (!taken[j]) rest.push_back(j);
        const int64_t extra = need - int64_t(cand.size());
        partial_shuffle(rest, extra, stream_key(st.prm.seed, kSample, uint64_t(h)));
        cand.insert(cand.end(), rest.begin(), rest.begin() + extra);
    }
    return cand;
}

// Alg. 6 in postorder over every node except the root.  With sampler set,
// the sampled blocks K_{I'a} of a whole level are generated on the GPU in
// one call before the level's decompositions run on the host.
static void skeletonize(const Ctx& c, Structure& st, const std::vector<int64_t>& knn, int kappa,
                        DeviceSampler* sampler) {
    const int L = st.depth;
    st.skel.assign(st.n_nodes(), {});
    st.P.assign(st.n_nodes(), {});
    for (int lvl = L; lvl >= 1; --lvl) {
        const int64_t first = (int64_t(1) << lvl) - 1, cnt = int64_t(1) << lvl;
        if (sampler) {
            const size_t nc = static_cast<size_t>(cnt);
            std::vector<std::vector<int64_t>> rows(nc), cols(nc);
            std::vector<std::vector<double>> A(nc);
            parallel_for(cnt, c.par, [&](int64_t t) {
                const int64_t h = first + t;
                if (lvl == L) {
                    cols[t].assign(st.perm.begin() + st.node_off[h], st.perm.begin() + st.node_off[h] + st.node_size[h]);
                } else {
                    cols[t] = st.skel[2 * h + 1];
                    cols[t].insert(cols[t].end(), st.skel[2 * h + 2].begin(), st.skel[2 * h + 2].end());
                }
                rows[t] = sample_rows(st, knn, kappa, h);
                A[t].resize(rows[t].size() * cols[t].size());
            });
            // batches of about 8 M entries: the GPU samples batch b + 1
            // while the host decomposes batch b
            std::vector<std::pair<int64_t, int64_t>> batches;  // node ranges [t0, t1)
            for (int64_t t0 = 0; t0 < cnt;) {
                int64_t t1 = t0, e = 0;
                while (t1 < cnt && (t1 == t0 || e + int64_t(A[t1].size()) <= (int64_t(1) << 23))) e += int64_t(A[t1++].size());
                batches.emplace_back(t0, t1);
                t0 = t1;
            }
            auto jobs_of = [&](size_t b) {
                std::vector<SampleJob> jobs;
                for (int64_t t = batches[b].first; t < batches[b].second; ++t)
                    jobs.push_back(SampleJob{rows[t].data(), int64_t(rows[t].size()), cols[t].data(),
                                             int64_t(cols[t].size()), nullptr});
                return jobs;
            };
            int slot = sampler->submit(jobs_of(0));
            for (size_t b = 0; b < batches.size(); ++b) {
                const std::vector<const double*> blk = sampler->wait(slot);
                if (b + 1 < batches.size()) slot = sampler->submit(jobs_of(b + 1));
                const int64_t t0 = batches[b].first;
                parallel_for(batches[b].second - t0, c.par, [&](int64_t u) {
                    const int64_t t = t0 + u, h = first + t;
                    const int64_t m = int64_t(rows[t].size()), n = int64_t(cols[t].size());
                    std::copy(blk[size_t(u)], blk[size_t(u)] + m * n, A[t].begin());
                    IdResult id = interpolative_decomposition(A[t], m, n, st.prm.s, st.prm.tau);
                    std::vector<int64_t> sk(id.s);
                    for (int64_t v = 0; v < id.s; ++v) sk[v] = cols[t][id.perm[v]];
                    st.skel[h] = std::move(sk);
                    st.P[h] = std::move(id.P);
                    std::vector<double>().swap(A[t]);
                });
            }
            continue;
        }
        parallel_for(cnt, c.par, [&](int64_t t) {
            const int64_t h = first + t;
            std::vector<int64_t> cols;
            if (lvl == L) {
                cols.assign(st.perm.begin() + st.node_off[h], st.perm.begin() + st.node_off[h] + st.node_size[h]);
            } else {
                cols = st.skel[2 * h + 1];
                cols.insert(cols.end(), st.skel[2 * h + 2].begin(), st.skel[2 * h + 2].end());
            }
            const std::vector<int64_t> rows = sample_rows(st, knn, kappa, h);
            const int64_t m = int64_t(rows.size()), n = int64_t(cols.size());
            std::vector<double> Arm(size_t(m * n)), A(size_t(m * n));
            c.K.block(rows.data(), m, cols.data(), n, Arm.data());
            for (int64_t i = 0; i < m; ++i)
                for (int64_t j = 0; j < n; ++j) A[size_t(j * m + i)] = Arm[size_t(i * n + j)];
            IdResult id = interpolative_decomposition(A, m, n, st.prm.s, st.prm.tau);
            std::vector<int64_t> sk(id.s);
            for (int64_t u = 0; u < id.s; ++u) sk[u] = cols[id.perm[u]];
            st.skel[h] = std::move(sk);
            st.P[h] = std::move(id.P);
        });
    }
}

void cache_blocks_host(const Entries& K, Structure& st) {
    const int64_t nl = st.n_leaves();
    const bool par = K.is_generator();
    st.near_blocks.assign(nl, {});
    parallel_for(nl, par, [&](int64_t b) {
        const int64_t hb = st.leaf_node(b);
        const int64_t* rb = &st.perm[st.node_off[hb]];
        for (int64_t a : st.near[b]) {
            const int64_t ha = st.leaf_node(a);
            std::vector<double> blk(size_t(st.node_size[hb] * st.node_size[ha]));
            K.block(rb, st.node_size[hb], &st.perm[st.node_off[ha]], st.node_size[ha], blk.data());
            st.near_blocks[b].push_back(std::move(blk));
        }
    });
    st.far_blocks.assign(st.n_nodes(), {});
    parallel_for(st.n_nodes(), par, [&](int64_t h) {
        for (int64_t a : st.far[h]) {
            std::vector<double> blk(st.skel[h].size() * st.skel[a].size());
            K.block(st.skel[h].data(), int64_t(st.skel[h].size()), st.skel[a].data(),
                    int64_t(st.skel[a].size()), blk.data());
            st.far_blocks[h].push_back(std::move(blk));
        }
    });
}

void compress(const Entries& K, Structure& st) {
    const auto t0 = std::chrono::steady_clock::now();
    const Params& prm = st.prm;
    // a user callback is called from one thread at a time
    const bool par = K.is_generator();
    if (prm.num_threads > 0) omp_set_num_threads(prm.num_threads);
    Ctx c{K, prm, std::vector<double>(size_t(K.n)), par};
    parallel_for((K.n + 1023) / 1024, par, [&](int64_t blk) {
        for (int64_t i = blk * 1024; i < std::min<int64_t>(K.n, (blk + 1) * 1024); ++i) c.diagK[i] = K.diag(i);
    });
    st.n = K.n;
    const int kappa = int(std::min<int64_t>(prm.kappa, K.n));
    std::vector<int64_t> knn = all_nearest_neighbors(c, st.ann_iters, st.ann_recall);
    auto nodes = build_tree(c, 0, 0);
    st.depth = tree_depth(K.n, prm.m);
    const int64_t nl = st.n_leaves();
    st.perm.clear();
    st.node_size.assign(st.n_nodes(), 0);
    std::vector<int64_t> leaf_of(K.n);
    for (int64_t b = 0; b < nl; ++b) {
        const auto& lf = nodes[st.leaf_node(b)];
        st.node_size[st.leaf_node(b)] = int64_t(lf.size());
        for (int64_t i : lf) leaf_of[i] = b;
        st.perm.insert(st.perm.end(), lf.begin(), lf.end());
    }
    fill_node_extents(st);
    leaf_near(st, knn, kappa, leaf_of);
    if (prm.far_mode == GOFMM_FAR_PAPER) far_paper(st);
    else far_symmetric(st);
    std::unique_ptr<DeviceSampler> sampler;
    if (prm.sample_device) sampler = std::make_unique<DeviceSampler>(K, prm.device);
    skeletonize(c, st, knn, kappa, sampler.get());
    if (!K.is_generator() && prm.cache_mode == GOFMM_CACHE_BLOCKS) cache_blocks_host(K, st);
    st.compress_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace gofmm
