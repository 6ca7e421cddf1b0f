// Tensor-core (tcgen05) forms of the Gaussian stage and of the final pass.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

struct lev_handle;

namespace lev {

// Handle services used by the tensor-core module (defined in api.cu). Scratch slots: 0 operand
// image of the final pass, 1 split-K partials, 2 operand B^T of the Gaussian stage, 3 padded A.
int handle_scratch(lev_handle* h, int which, size_t bytes, void** out);
int handle_num_sms(lev_handle* h);
// The two events to record around the final pass kernel when the handle's timing is on, else null.
const cudaEvent_t* handle_final_marks(lev_handle* h);
int32_t* handle_status(lev_handle* h);
int handle_gaussian(lev_handle* h, int64_t m, int64_t s, uint64_t seed, int kind, cudaStream_t st,
                    const float** g32, const __nv_bfloat16** ghi);
int handle_fail(int code, const char* msg);

// A~ (m x d) = G B with prec in {LEV_TF32, LEV_BF16, LEV_BF16X3}.
int tc_gaussian_stage(lev_handle* h, const float* B, int64_t m, int64_t s, int64_t d, uint64_t seed,
                      int32_t prec, float* Atilde, cudaStream_t st);

// The K-major BF16 operand of the Gaussian stage blocked by 64 rows of B (img[g][c][k] =
// B[64 g + k][c], K padded to ld = s rounded up to 64), in scratch slot 2: hi, and lo for
// LEV_BF16X3 (null for LEV_BF16). LEV_EINVAL for the other precisions.
int tc_gaussian_operand(lev_handle* h, int64_t s, int64_t d, int32_t prec, __nv_bfloat16** hi, __nv_bfloat16** lo,
                        int64_t* ld);
// A~ = G B with B already written as that operand (prec LEV_BF16 or LEV_BF16X3).
int tc_gaussian_stage_blocked(lev_handle* h, int64_t m, int64_t s, int64_t d, uint64_t seed, int32_t prec,
                              float* Atilde, cudaStream_t st);

// theta = rowsum((A Mfull)^2) with prec in {LEV_TF32, LEV_BF16, LEV_BF16X3}.
int tc_final_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, const float* Mfull,
                   int64_t k, int32_t prec, float* theta, cudaStream_t st);

}  // namespace lev
