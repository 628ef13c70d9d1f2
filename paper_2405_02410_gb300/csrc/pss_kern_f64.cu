// FP64 instantiation of the auxiliary kernels and of the step kernels with
// radix-8 FFT passes (double fields, double2 spectra).
#include "pss_kernels.cuh"
namespace pss {
PSS_INSTANTIATE_AUX(double)
PSS_INSTANTIATE_STEP(double, 8)
}
