// signature_tc.cu -- placeholder until the tcgen05 path lands.
#include "common.cuh"

namespace aptidx {

bool tc_supported(Ctx*) { return false; }

int prepare_tc(Ctx* c) {
    return set_error(c, APTIDX_E_INVALID_ARG, "tensor-core path not built yet");
}

cudaError_t launch_signatures_tc(Ctx*, float*, uint16_t*, uint16_t*, int64_t) {
    return cudaErrorNotSupported;
}

}  // namespace aptidx
