// The persistent FP32 2D step of a KPZ field (mode 1: the gradient-square
// term), in a translation unit of its own so that nvcc builds it in parallel.
#include "pss_persist2d.cuh"
namespace pss {

template <int N, int E, int NNW>
cudaError_t launch_p2k_ne(const P2Args &a, int nblocks, cudaStream_t st) {
    using L = P2Shape<N, E, NNW>;
    cudaError_t e = ensure_smem(k2p_step<N, E, NNW, 1>, L::BYTES);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks, 1, 1);
    cfg.blockDim = dim3(L::THREADS, 1, 1);
    cfg.dynamicSmemBytes = L::BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // every CTA resident at once (grid barriers)
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k2p_step<N, E, NNW, 1>, a);
}

cudaError_t launch_p2_kpz(const P2Args &a, int n, int E, int nblocks, cudaStream_t st) {
    switch (n) {
        case 256: return E == 16 ? launch_p2k_ne<256, 16, 4>(a, nblocks, st) : launch_p2k_ne<256, 8, 4>(a, nblocks, st);
        case 512: return E == 16 ? launch_p2k_ne<512, 16, 4>(a, nblocks, st) : launch_p2k_ne<512, 8, 4>(a, nblocks, st);
        case 1024:
            return E == 16 ? launch_p2k_ne<1024, 16, 4>(a, nblocks, st) : launch_p2k_ne<1024, 8, 4>(a, nblocks, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pss
