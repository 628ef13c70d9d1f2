// FP32 2D step kernels with one FFT group per transform (sides of 256, 512 or 1024 points).
#include "pss_adj2d.cuh"
namespace pss {

// a.E: radix of the FFT passes, 8 or 16 (or 32 for sides of 1024); a radix a
// side does not take falls back to 16
cudaError_t launch_col2(const ColArgs<float> &a, int nslots, int ntiles, cudaStream_t st) {
    const bool r16 = a.E == 16;
    switch (a.sp.n_inner) {
        case 256: return r16 ? launch_col2_ne<256, 16>(a, nslots, ntiles, st) : launch_col2_ne<256, 8>(a, nslots, ntiles, st);
        case 512: return r16 ? launch_col2_ne<512, 16>(a, nslots, ntiles, st) : launch_col2_ne<512, 8>(a, nslots, ntiles, st);
        case 1024:
            return a.E == 32 ? launch_col2_ne<1024, 32>(a, nslots, ntiles, st)
                 : r16       ? launch_col2_ne<1024, 16>(a, nslots, ntiles, st)
                             : launch_col2_ne<1024, 8>(a, nslots, ntiles, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_row2(const RowArgs<float> &a, int nslots, cudaStream_t st, bool tiled) {
    const bool r16 = a.E == 16;
#define PSS_ROW2(N, E)                                                                                    \
    (!tiled ? launch_row2_ne<N, E, false, false>(a, nslots, st)                                           \
            : (a.mode == ROW_ADJ ? launch_row2_ne<N, E, true, true>(a, nslots, st)                        \
                                 : launch_row2_ne<N, E, true, false>(a, nslots, st)))
    switch (a.sp.nx) {
        case 256: return r16 ? PSS_ROW2(256, 16) : PSS_ROW2(256, 8);
        case 512: return r16 ? PSS_ROW2(512, 16) : PSS_ROW2(512, 8);
        case 1024: return a.E == 32 ? PSS_ROW2(1024, 32) : r16 ? PSS_ROW2(1024, 16) : PSS_ROW2(1024, 8);
        default: return cudaErrorInvalidValue;
    }
#undef PSS_ROW2
}

// the adjoint's column part (modes COL_ADJ_A, COL_ADJ_B, COL_ADJ_BA) on FFT
// groups: a.E the pass radix (8 or 16), one column pair per CTA
cudaError_t launch_col2_adj(const ColArgs<float> &a, int nslots, cudaStream_t st) {
    const bool r16 = a.E == 16;
    switch (a.sp.ny) {
        case 256: return r16 ? launch_col2_adj_ne<256, 16>(a, nslots, st) : launch_col2_adj_ne<256, 8>(a, nslots, st);
        case 512: return r16 ? launch_col2_adj_ne<512, 16>(a, nslots, st) : launch_col2_adj_ne<512, 8>(a, nslots, st);
        case 1024: return r16 ? launch_col2_adj_ne<1024, 16>(a, nslots, st) : launch_col2_adj_ne<1024, 8>(a, nslots, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pss
