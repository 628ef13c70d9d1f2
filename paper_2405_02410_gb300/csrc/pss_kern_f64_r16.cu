// FP64 instantiation of the step kernels with radix-16 FFT passes (double fields, double2 spectra).
#include "pss_kernels.cuh"
namespace pss {
PSS_INSTANTIATE_STEP(double, 16)
}
