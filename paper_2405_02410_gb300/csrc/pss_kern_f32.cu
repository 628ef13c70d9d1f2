// FP32 instantiation of the step kernels (float fields, float2 spectra).
#include "pss_kernels.cuh"
namespace pss {
PSS_INSTANTIATE(float)
}
