// FP32 instantiation of the step kernels with radix-16 FFT passes (float fields, float2 spectra).
#include "pss_kernels.cuh"
namespace pss {
PSS_INSTANTIATE_STEP(float, 16)
}
