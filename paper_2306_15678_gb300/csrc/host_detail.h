// host_detail.h -- host helpers shared by the C ABI translation units (not
// part of the ABI; hidden from the library's exported symbols).
#pragma once
#include <cuda_runtime.h>

#include "../../include/nlse.h"
#include "kernels.cuh"

#define NLSE_HIDDEN __attribute__((visibility("hidden")))

namespace nlse {
namespace detail {

// FP32 propagator tables for p into px/py and, when tw is non-null, the FP32
// pass-major twiddle table for n: kDither dithered copies of n entries each
// (copy k mod kDither serves step k); synchronises s.
NLSE_HIDDEN nlse_status upload_tables_f32(const nlse_params* p, cudaStream_t s, unsigned char* px,
                                          unsigned char* py, unsigned char* tw);
// FP32 screen coefficients of p (Eq. 3, gains theta)
NLSE_HIDDEN ScreenCoef<float> screen_coef_f32(const nlse_params* p);
// global phase factor of step k (0-based) in FP32, as a single grid applies
// it, and in *applied (may be null) the angle it turns the field by
NLSE_HIDDEN float2 rot_step_f32(long long k, double* applied);
// deterministic FP64 reduction of nparts (sum, max) partials into out[0..1]
NLSE_HIDDEN cudaError_t finalize(const double* partials, int nparts, double scale, double* out, int* status,
                                 cudaStream_t s);

}  // namespace detail
}  // namespace nlse
