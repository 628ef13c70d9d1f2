// The backward pass of a recomputed segment of the FP32 2D adjoint (square
// sides of 256, 512 or 1024 points): one cooperative launch of k2p_adj.
#include "pss_persist_adj.cuh"
namespace pss {

template <int N, int E>
cudaError_t launch_p2_adj_ne(const P2AdjArgs &a, int nblocks, cudaStream_t st) {
    using L = P2AdjShape<N, E>;
    cudaError_t e = ensure_smem(k2p_adj<N, E>, L::BYTES);
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
    return cudaLaunchKernelEx(&cfg, k2p_adj<N, E>, a);
}

cudaError_t launch_p2_adj(const P2AdjArgs &a, int n, int E, int nblocks, cudaStream_t st) {
    // a CTA holds at most 2 of the (n / 2 + 2) / 2 column pairs and 4 of the n / 2 row pairs
    const int uc = (n / 2 + 2) / 2;
    if (nblocks < (uc + 1) / 2 || nblocks < n / 8 || a.len < 1) return cudaErrorInvalidConfiguration;
    switch (n) {
        case 256: return E == 16 ? launch_p2_adj_ne<256, 16>(a, nblocks, st) : launch_p2_adj_ne<256, 8>(a, nblocks, st);
        case 512: return E == 16 ? launch_p2_adj_ne<512, 16>(a, nblocks, st) : launch_p2_adj_ne<512, 8>(a, nblocks, st);
        case 1024:
            return E == 16 ? launch_p2_adj_ne<1024, 16>(a, nblocks, st) : launch_p2_adj_ne<1024, 8>(a, nblocks, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pss
