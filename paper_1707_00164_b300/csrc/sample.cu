// Entry generation on the GPU for compression: the sampled blocks K_{I'a}
// that every interpolative decomposition factors (Alg. 2 steps 8-9), for
// all nodes of a tree level in one launch.  Entries are computed in FP64
// with the generator's formula and coordinate order (Gaussian
// exp(-|x_i - x_j|^2 / (2 h^2)), inverse multiquadric
// 1 / sqrt(1 + |x_i - x_j|^2 / h^2), plus the shift when i = j) and written
// column-major, the layout the host's pivoted QR reads.  The pivoted QR and
// the triangular solve stay on the host in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "eval_state.hpp"
#include "gofmm_internal.hpp"

namespace gofmm {
namespace {

struct SampleDesc {
    int64_t roff, coff;  // offsets of the row / column index lists in idx[]
    int64_t out;         // first element of the block in the output buffer
    int32_t m, n;
};

__global__ void sample_blocks_kernel(const SampleDesc* __restrict__ jobs, const int64_t* __restrict__ idx,
                                     const double* __restrict__ pts, int dim, int kind, double h, double shift,
                                     double* __restrict__ out) {
    const SampleDesc b = jobs[blockIdx.x];
    const int64_t total = int64_t(b.m) * b.n;
    const double two_h2 = 2.0 * h * h, h2 = h * h;
    for (int64_t e = int64_t(blockIdx.y) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.y) * blockDim.x) {
        const int64_t j = e / b.m, i = e % b.m;  // column-major: consecutive threads share a column
        const int64_t ri = idx[b.roff + i], cj = idx[b.coff + j];
        // squared distance coordinate by coordinate without fused
        // multiply-adds, as the host generator accumulates it
        double acc = 0.0;
        for (int d = 0; d < dim; ++d) {
            const double t = __dsub_rn(pts[ri * dim + d], pts[cj * dim + d]);
            acc = __dadd_rn(acc, __dmul_rn(t, t));
        }
        double v = kind == GOFMM_GEN_GAUSSIAN ? exp(-(acc / two_h2)) : 1.0 / sqrt(1.0 + acc / h2);
        if (ri == cj) v += shift;
        out[b.out + e] = v;
    }
}

}  // namespace

// One buffer set of the asynchronous path: descriptors and index lists
// (pinned, uploaded), the blocks (device, then pinned), and the event that
// marks them landed.
struct DeviceSampler::Slot {
    SampleDesc* h_desc = nullptr;
    int64_t* h_idx = nullptr;
    double* h_out = nullptr;
    SampleDesc* d_desc = nullptr;
    int64_t* d_idx = nullptr;
    double* d_out = nullptr;
    size_t cap_desc = 0, cap_idx = 0, cap_out = 0;
    cudaEvent_t done = nullptr;
    std::vector<int64_t> offs;
};

DeviceSampler::DeviceSampler(const Entries& K, int device) : K_(K), device_(device) {
    if (!K.is_generator()) fail(GOFMM_ERR_ARG, "device sampling needs a generator kind (Gaussian or IMQ)");
    DeviceGuard g(device_);
    d_pts_ = dupload(K.pts);
    cudaStream_t s = nullptr;
    CUDA_OK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    stream_ = s;
    for (Slot*& sl : slots_) {
        sl = new Slot();
        CUDA_OK(cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming));
    }
}

DeviceSampler::~DeviceSampler() {
    int old = -1;
    cudaGetDevice(&old);
    cudaSetDevice(device_);
    if (stream_) cudaStreamSynchronize(static_cast<cudaStream_t>(stream_));
    for (Slot* sl : slots_) {
        if (!sl) continue;
        if (sl->h_desc) cudaFreeHost(sl->h_desc);
        if (sl->h_idx) cudaFreeHost(sl->h_idx);
        if (sl->h_out) cudaFreeHost(sl->h_out);
        dfree(sl->d_desc);
        dfree(sl->d_idx);
        dfree(sl->d_out);
        if (sl->done) cudaEventDestroy(sl->done);
        delete sl;
    }
    if (stream_) cudaStreamDestroy(static_cast<cudaStream_t>(stream_));
    dfree(d_pts_);
    if (old >= 0) cudaSetDevice(old);
}

int DeviceSampler::submit(const std::vector<SampleJob>& jobs) {
    DeviceGuard g(device_);
    const int id = next_;
    next_ ^= 1;
    Slot& sl = *slots_[id];
    CUDA_OK(cudaEventSynchronize(sl.done));  // the slot's previous batch was consumed
    size_t n_idx = 0, n_out = 0;
    for (const SampleJob& jb : jobs) {
        n_idx += size_t(jb.m + jb.n);
        n_out += size_t(jb.m * jb.n);
    }
    auto grow_host = [](auto*& p, size_t& cap, size_t need) {
        if (need <= cap) return;
        if (p) CUDA_OK(cudaFreeHost(p));
        p = nullptr;
        CUDA_OK(cudaMallocHost(reinterpret_cast<void**>(&p), need * sizeof(*p)));
        cap = need;
    };
    size_t c1 = sl.cap_desc, c2 = sl.cap_idx, c3 = sl.cap_out;
    grow_host(sl.h_desc, c1, std::max<size_t>(jobs.size(), 1));
    grow_host(sl.h_idx, c2, std::max<size_t>(n_idx, 1));
    grow_host(sl.h_out, c3, std::max<size_t>(n_out, 1));
    if (c1 > sl.cap_desc) { dfree(sl.d_desc); sl.d_desc = dalloc<SampleDesc>(c1); }
    if (c2 > sl.cap_idx) { dfree(sl.d_idx); sl.d_idx = dalloc<int64_t>(c2); }
    if (c3 > sl.cap_out) { dfree(sl.d_out); sl.d_out = dalloc<double>(c3); }
    sl.cap_desc = c1;
    sl.cap_idx = c2;
    sl.cap_out = c3;
    sl.offs.assign(jobs.size(), 0);
    size_t pi = 0, po = 0;
    for (size_t k = 0; k < jobs.size(); ++k) {
        const SampleJob& jb = jobs[k];
        for (int64_t t = 0; t < jb.m; ++t)
            if (jb.rows[t] < 0 || jb.rows[t] >= K_.n) fail(GOFMM_ERR_ARG, "sample row out of range");
        for (int64_t t = 0; t < jb.n; ++t)
            if (jb.cols[t] < 0 || jb.cols[t] >= K_.n) fail(GOFMM_ERR_ARG, "sample column out of range");
        SampleDesc d{};
        d.roff = int64_t(pi);
        std::copy(jb.rows, jb.rows + jb.m, sl.h_idx + pi);
        pi += size_t(jb.m);
        d.coff = int64_t(pi);
        std::copy(jb.cols, jb.cols + jb.n, sl.h_idx + pi);
        pi += size_t(jb.n);
        d.out = int64_t(po);
        d.m = int32_t(jb.m);
        d.n = int32_t(jb.n);
        sl.h_desc[k] = d;
        sl.offs[k] = int64_t(po);
        po += size_t(jb.m * jb.n);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    if (!jobs.empty() && po > 0) {
        CUDA_OK(cudaMemcpyAsync(sl.d_desc, sl.h_desc, jobs.size() * sizeof(SampleDesc), cudaMemcpyHostToDevice, s));
        CUDA_OK(cudaMemcpyAsync(sl.d_idx, sl.h_idx, pi * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        dim3 grid(unsigned(jobs.size()), 16);
        sample_blocks_kernel<<<grid, 256, 0, s>>>(sl.d_desc, sl.d_idx, d_pts_, K_.dim, K_.kind, K_.h, K_.shift,
                                                  sl.d_out);
        CUDA_OK(cudaGetLastError());
        CUDA_OK(cudaMemcpyAsync(sl.h_out, sl.d_out, po * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    CUDA_OK(cudaEventRecord(sl.done, s));
    return id;
}

std::vector<const double*> DeviceSampler::wait(int slot) {
    DeviceGuard g(device_);
    Slot& sl = *slots_[slot];
    CUDA_OK(cudaEventSynchronize(sl.done));
    std::vector<const double*> out(sl.offs.size());
    for (size_t k = 0; k < out.size(); ++k) out[k] = sl.h_out + sl.offs[k];
    return out;
}

void DeviceSampler::sample(const std::vector<SampleJob>& jobs) {
    if (jobs.empty()) return;
    DeviceGuard g(device_);
    // batches of at most ~32 M entries (256 MB) on the device at once
    constexpr int64_t kBatch = int64_t(1) << 25;
    size_t j0 = 0;
    while (j0 < jobs.size()) {
        std::vector<SampleDesc> desc;
        std::vector<int64_t> idx;
        int64_t entries = 0;
        size_t j1 = j0;
        while (j1 < jobs.size() && (j1 == j0 || entries + jobs[j1].m * jobs[j1].n <= kBatch)) {
            const SampleJob& jb = jobs[j1];
            SampleDesc d{};
            d.roff = int64_t(idx.size());
            idx.insert(idx.end(), jb.rows, jb.rows + jb.m);
            d.coff = int64_t(idx.size());
            idx.insert(idx.end(), jb.cols, jb.cols + jb.n);
            d.out = entries;
            d.m = int32_t(jb.m);
            d.n = int32_t(jb.n);
            for (int64_t t = 0; t < jb.m; ++t)
                if (jb.rows[t] < 0 || jb.rows[t] >= K_.n) fail(GOFMM_ERR_ARG, "sample row out of range");
            for (int64_t t = 0; t < jb.n; ++t)
                if (jb.cols[t] < 0 || jb.cols[t] >= K_.n) fail(GOFMM_ERR_ARG, "sample column out of range");
            entries += jb.m * jb.n;
            desc.push_back(d);
            ++j1;
        }
        if (entries > 0) {
            SampleDesc* d_desc = dupload(desc);
            int64_t* d_idx = dupload(idx);
            double* d_out = dalloc<double>(size_t(entries));
            dim3 grid(unsigned(desc.size()), 16);
            sample_blocks_kernel<<<grid, 256>>>(d_desc, d_idx, d_pts_, K_.dim, K_.kind, K_.h, K_.shift, d_out);
            const cudaError_t le = cudaGetLastError();
            std::vector<double> host(static_cast<size_t>(entries));
            const cudaError_t ce =
                le == cudaSuccess ? cudaMemcpy(host.data(), d_out, host.size() * sizeof(double), cudaMemcpyDeviceToHost)
                                  : le;
            dfree(d_desc);
            dfree(d_idx);
            dfree(d_out);
            CUDA_OK(ce);
            for (size_t k = j0; k < j1; ++k)
                std::copy(host.begin() + desc[k - j0].out, host.begin() + desc[k - j0].out + jobs[k].m * jobs[k].n,
                          jobs[k].out);
        }
        j0 = j1;
    }
}

}  // namespace gofmm
