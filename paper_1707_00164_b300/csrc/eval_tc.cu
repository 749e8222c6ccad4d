// Tensor-core evaluation path (TF32 / BF16 / split-BF16x3 on sm_103a).
#include "eval_state.hpp"

namespace gofmm {

struct TcState {};

void tc_prepare(Handle&, DeviceState&, int64_t, int) {
    fail(GOFMM_ERR_UNSUPPORTED, "tensor-core precisions are not built in this library version");
}
bool tc_ready(const DeviceState&, int64_t, int) { return false; }
int tc_run(Handle&, DeviceState&, const float*, int64_t, float*, int64_t, int, int, cudaStream_t) {
    fail(GOFMM_ERR_UNSUPPORTED, "tensor-core precisions are not built in this library version");
}
void tc_destroy(DeviceState& D) {
    delete D.tc;
    D.tc = nullptr;
}

}  // namespace gofmm
