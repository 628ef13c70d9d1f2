// The persistent FP32 2D step (square sides of 256, 512 or 1024 points):
// one cooperative launch of k2p_step per run of steps.
#include "pss_persist2d.cuh"
namespace pss {

template <int N, int E, int NNW, int MODE>
cudaError_t launch_p2_ne(const P2Args &a, int nblocks, cudaStream_t st) {
    using L = P2Shape<N, E, NNW>;
    cudaError_t e = ensure_smem(k2p_step<N, E, NNW, MODE>, L::BYTES);
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
    return cudaLaunchKernelEx(&cfg, k2p_step<N, E, NNW, MODE>, a);
}

cudaError_t launch_p2(const P2Args &a, int n, int E, int nblocks, int mode, cudaStream_t st) {
    // a CTA holds at most 2 of the (n / 2 + 2) / 2 column pairs and 4 of the n / 2 row pairs
    const int uc = (n / 2 + 2) / 2;
    if (nblocks < (uc + 1) / 2 || nblocks < n / 8 || a.nsteps < 1) return cudaErrorInvalidConfiguration;
    if (mode == 1) return launch_p2_kpz(a, n, E, nblocks, st);
    // beside the FFT groups, 4 noise warps (the register budget of 168 per
    // thread that leaves the radix-16 transforms measured faster than 8 warps)
    switch (n) {
        case 256: return E == 16 ? launch_p2_ne<256, 16, 4, 0>(a, nblocks, st) : launch_p2_ne<256, 8, 4, 0>(a, nblocks, st);
        case 512: return E == 16 ? launch_p2_ne<512, 16, 4, 0>(a, nblocks, st) : launch_p2_ne<512, 8, 4, 0>(a, nblocks, st);
        case 1024:
            return E == 16 ? launch_p2_ne<1024, 16, 4, 0>(a, nblocks, st) : launch_p2_ne<1024, 8, 4, 0>(a, nblocks, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pss
