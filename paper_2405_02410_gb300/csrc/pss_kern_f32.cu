// FP32 instantiation of the auxiliary kernels and of the step kernels with
// radix-8 FFT passes (float fields, float2 spectra).
#include "pss_kernels.cuh"
namespace pss {
PSS_INSTANTIATE_AUX(float)
PSS_INSTANTIATE_STEP(float, 8)
}
