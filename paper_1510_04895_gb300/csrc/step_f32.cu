// Instantiations of the fused Chebyshev step kernel for float vectors.
#include "filter_kernels.cuh"

namespace chebfd {

namespace {

template <bool CPLX, int G, int CPT>
void launch_g(const SellView& H, StepMode mode, const StepArgs& a, int wc,
              int grid, cudaStream_t s) {
    constexpr int SLOTS = STEP_THREADS / G;
    constexpr int CPC = CPLX ? ChunkT<float>::K / 2 : ChunkT<float>::K;
    (void)CPC;
    const size_t smem = a.moments ? (size_t)SLOTS * 2 * a.nb * sizeof(double) : 0;
    switch (mode) {
        case MODE_SPMV:
            cheb_step_kernel<float, CPLX, G, CPT, MODE_SPMV><<<grid, STEP_THREADS, smem, s>>>(H, a, wc);
            break;
        case MODE_SECOND:
            cheb_step_kernel<float, CPLX, G, CPT, MODE_SECOND><<<grid, STEP_THREADS, smem, s>>>(H, a, wc);
            break;
        case MODE_STEP:
            cheb_step_kernel<float, CPLX, G, CPT, MODE_STEP><<<grid, STEP_THREADS, smem, s>>>(H, a, wc);
            break;
    }
}

template <bool CPLX>
void launch_c(const SellView& H, StepMode mode, const StepArgs& a, int wc, int grid,
              cudaStream_t s) {
    if (wc > 32) launch_g<CPLX, 32, 2>(H, mode, a, wc, grid, s);
    else if (wc > 16) launch_g<CPLX, 32, 1>(H, mode, a, wc, grid, s);
    else if (wc > 8) launch_g<CPLX, 16, 1>(H, mode, a, wc, grid, s);
    else if (wc > 4) launch_g<CPLX, 8, 1>(H, mode, a, wc, grid, s);
    else if (wc > 2) launch_g<CPLX, 4, 1>(H, mode, a, wc, grid, s);
    else if (wc > 1) launch_g<CPLX, 2, 1>(H, mode, a, wc, grid, s);
    else launch_g<CPLX, 1, 1>(H, mode, a, wc, grid, s);
}

}  // namespace

void launch_step_f32(const SellView& H, bool cplx, StepMode mode, const StepArgs& a, int wc,
                    int grid, cudaStream_t s) {
    if (cplx) launch_c<true>(H, mode, a, wc, grid, s);
    else launch_c<false>(H, mode, a, wc, grid, s);
}

}  // namespace chebfd
