// gofmm_evaluate_static: the FP64 / FP32 evaluation with its scratch in a
// fixed device array instead of handle-allocated buffers.
//
// It serves callers that must not allocate device memory once they are
// running: a serving loop that reserved its whole memory budget at start-up
// and may not grow it per request (a cudaMalloc there can fail, and it also
// synchronises the device, stalling every request in flight), or host code
// that lives under another framework's caching allocator that owns the free
// memory.  Such a caller prepares the handle once (gofmm_prepare, which does
// allocate), then evaluates through this entry point without any further
// allocation.
//
// The scratch is the file-scope array below: kStaticScratchBytes (32 MiB) on
// every device that loads this library, held until the process exits.  In
// host code the array's name only stands in for the device symbol, so the
// device address is looked up with cudaGetSymbolAddress, once per device,
// with that device current, on the first call on that device (make that
// first call before any stream capture).  Every call shares the array and it
// keeps the previous call's contents; the evaluation writes every scratch
// element it later reads, so nothing has to be cleared, but calls whose
// executions overlap on the GPU (other streams, other handles) race on it.
#include <mutex>
#include <unordered_map>

#include "eval_state.hpp"

namespace gofmm {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {
std::mutex g_scratch_mu;
std::unordered_map<int, void*> g_scratch_addr;  // device -> address of g_static_scratch

void* static_scratch(int device) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    auto it = g_scratch_addr.find(device);
    if (it != g_scratch_addr.end()) return it->second;
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr)
        fail(GOFMM_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[device] = p;
    return p;
}

size_t round_up(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

void device_evaluate_static(Handle& H, const void* W, int64_t ldw, void* U, int64_t ldu, int64_t r, int dtype,
                            int precision, void* stream) {
    if (!W || !U) fail(GOFMM_ERR_ARG, "W and U must not be NULL");
    // the same bound on r as gofmm_evaluate: the scratch sizes below are
    // products with r and must not wrap, and the kernels take r as an int
    if (r < 1 || r > (int64_t(1) << 30)) fail(GOFMM_ERR_ARG, "r must be in [1, 2^30]");
    if (ldw < r || ldu < r) fail(GOFMM_ERR_ARG, "leading dimensions must be >= r");
    if (precision != GOFMM_PREC_FP64 && precision != GOFMM_PREC_FP32)
        fail(GOFMM_ERR_UNSUPPORTED, "the static-scratch evaluation supports FP64 and FP32 only");
    if ((precision == GOFMM_PREC_FP64) != (dtype == GOFMM_DTYPE_F64))
        fail(GOFMM_ERR_UNSUPPORTED, "FP64 precision needs F64 data and FP32 precision F32 data");
    const int fi = precision == GOFMM_PREC_FP64 ? 0 : 1;
    if (!H.dev || !H.dev->fam[fi].stores)
        fail(GOFMM_ERR_ARG, "handle not prepared for this precision: call gofmm_prepare first");
    const size_t es = precision == GOFMM_PREC_FP64 ? 8 : 4;
    const size_t wt = round_up(size_t(H.dev->n) * size_t(r) * es);
    const size_t sk = round_up(size_t(std::max<int64_t>(H.dev->S_tot, 1)) * size_t(r) * es);
    const size_t need = wt + 2 * sk;
    if (need > kStaticScratchBytes)
        fail(GOFMM_ERR_ARG, "evaluation needs " + std::to_string(need) + " bytes of scratch; the static scratch "
                            "holds " + std::to_string(kStaticScratchBytes) + " (use gofmm_evaluate)");
    DeviceGuard g(H.st.prm.device);
    char* base = static_cast<char*>(static_scratch(H.st.prm.device));
    simt_evaluate_on(H, W, ldw, U, ldu, int(r), precision, static_cast<cudaStream_t>(stream), base, base + wt,
                     base + wt + sk);
}

}  // namespace gofmm
