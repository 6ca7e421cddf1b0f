// Tensor-core forms (placeholder until the tcgen05 kernels land).
#include "lev_common.cuh"
#include "lev_tc.cuh"

namespace lev {

int tc_gaussian_stage(lev_handle*, const float*, int64_t, int64_t, int64_t, uint64_t, int32_t, float*,
                      cudaStream_t) {
    return handle_fail(LEV_EINVAL, "tensor-core Gaussian stage not available");
}

int tc_final_dense(lev_handle*, const float*, int64_t, int64_t, int64_t, const float*, int64_t, int32_t,
                   float*, cudaStream_t) {
    return handle_fail(LEV_EINVAL, "tensor-core final pass not available");
}

}  // namespace lev
