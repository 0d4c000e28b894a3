// Instantiations of the fused Chebyshev step kernel for double vectors.
#include <algorithm>
#include <cstdlib>

#include "filter_kernels.cuh"

namespace chebfd {

namespace {

// Resident blocks per SM of one instantiation (occupancy API, cached per
// kernel), capped by CHEBFD_STEP_BPS when set: the persistent grid is whole waves.
template <class Kern>
int blocks_per_sm(Kern kern, size_t smem) {
    int b = cached_occupancy(reinterpret_cast<const void*>(kern), STEP_THREADS, smem);
    if (const char* e = getenv("CHEBFD_STEP_BPS")) b = std::max(1, std::min(b, atoi(e)));
    return std::min(b, 8);
}

template <bool CPLX, int G, int CPT, int MODE, int L, bool ENS>
void launch_l(const SellView& H, const StepArgs& a, int wc, int sms, cudaStream_t s) {
    constexpr int SLOTS = STEP_THREADS / G;
    const size_t smem = a.moments ? (size_t)SLOTS * 2 * a.nb * sizeof(double) : 0;
    auto kern = cheb_step_kernel<double, CPLX, G, CPT, MODE, L, ENS>;
    const int grid = sms * blocks_per_sm(kern, a.moments ? (size_t)16384 : 0);
    kern<<<grid, STEP_THREADS, smem, s>>>(H, a, wc);
}

// Fixed-width kernels exist for the two row widths of the paper's matrices
// (N_nzr = 13 insulator, 4 graphene, Sec. 4); other widths take the generic path.
template <bool CPLX, int G, int CPT, int MODE>
void launch_m(const SellView& H, const StepArgs& a, int wc, int width, int sms,
              cudaStream_t s) {
    constexpr int L13 = CPT == 1 ? 13 : 0, L4 = CPT == 1 ? 4 : 0;
    if (a.coef != nullptr) {
        if (CPT == 1 && width == 13) launch_l<CPLX, G, CPT, MODE, L13, true>(H, a, wc, sms, s);
        else if (CPT == 1 && width == 4) launch_l<CPLX, G, CPT, MODE, L4, true>(H, a, wc, sms, s);
        else launch_l<CPLX, G, CPT, MODE, 0, true>(H, a, wc, sms, s);
        return;
    }
    if (CPT == 1 && width == 13) launch_l<CPLX, G, CPT, MODE, L13, false>(H, a, wc, sms, s);
    else if (CPT == 1 && width == 4) launch_l<CPLX, G, CPT, MODE, L4, false>(H, a, wc, sms, s);
    else launch_l<CPLX, G, CPT, MODE, 0, false>(H, a, wc, sms, s);
}

template <bool CPLX, int G, int CPT>
void launch_g(const SellView& H, StepMode mode, const StepArgs& a, int wc, int width, int sms,
              cudaStream_t s) {
    switch (mode) {
        case MODE_SPMV: launch_m<CPLX, G, CPT, MODE_SPMV>(H, a, wc, width, sms, s); break;
        case MODE_SECOND: launch_m<CPLX, G, CPT, MODE_SECOND>(H, a, wc, width, sms, s); break;
        case MODE_STEP: launch_m<CPLX, G, CPT, MODE_STEP>(H, a, wc, width, sms, s); break;
    }
}

template <bool CPLX>
void launch_c(const SellView& H, StepMode mode, const StepArgs& a, int wc, int width, int sms,
              cudaStream_t s) {
    if (wc > 32) launch_g<CPLX, 32, 2>(H, mode, a, wc, width, sms, s);
    else if (wc > 16) launch_g<CPLX, 32, 1>(H, mode, a, wc, width, sms, s);
    else if (wc > 8) launch_g<CPLX, 16, 1>(H, mode, a, wc, width, sms, s);
    else if (wc > 4) launch_g<CPLX, 8, 1>(H, mode, a, wc, width, sms, s);
    else if (wc > 2) launch_g<CPLX, 4, 1>(H, mode, a, wc, width, sms, s);
    else if (wc > 1) launch_g<CPLX, 2, 1>(H, mode, a, wc, width, sms, s);
    else launch_g<CPLX, 1, 1>(H, mode, a, wc, width, sms, s);
}

}  // namespace

void launch_step_f64(const SellView& H, bool cplx, StepMode mode, const StepArgs& a, int wc,
                    int width, int sms, cudaStream_t s) {
    if (cplx) launch_c<true>(H, mode, a, wc, width, sms, s);
    else launch_c<false>(H, mode, a, wc, width, sms, s);
}

}  // namespace chebfd
