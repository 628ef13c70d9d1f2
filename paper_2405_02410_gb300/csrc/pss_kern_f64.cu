// FP64 instantiation of the step kernels (double fields, double2 spectra).
#include "pss_kernels.cuh"
namespace pss {
PSS_INSTANTIATE(double)
}
