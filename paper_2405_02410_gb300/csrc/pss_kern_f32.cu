// FP32 instantiation of the auxiliary kernels and of the step kernels with
// radix-8 FFT passes (float fields, float2 spectra).
#include "pss_kernels.cuh"
namespace pss {
PSS_INSTANTIATE_AUX(float)

__global__ void k_set_i64(long long *dst, long long value) { *dst = value; }
cudaError_t launch_set_i64(long long *dst, long long value, cudaStream_t st) {
    k_set_i64<<<1, 1, 0, st>>>(dst, value);
    return cudaGetLastError();
}
PSS_INSTANTIATE_STEP(float, 8)
}
