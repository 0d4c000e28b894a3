// Launch of the double-float step kernel for one value type (complex or real);
// instantiated in df_step_c.cu and df_step_r.cu so the two compile in parallel.
#pragma once

#include <algorithm>

#include "df_kernels.cuh"

namespace chebfd {

template <bool CPLX, int G, int MODE>
void launch_df_gm(const SellView& H, const StepArgs& a, int wc, int width, int sms,
                  cudaStream_t s) {
    constexpr int LW = CPLX ? 13 : 4;  // row widths of the insulator and of graphene
    auto kern = width == LW ? cheb_df_kernel<CPLX, G, MODE, LW> : cheb_df_kernel<CPLX, G, MODE, 0>;
    const int grid =
        sms * std::min(8, cached_occupancy(reinterpret_cast<const void*>(kern), STEP_THREADS, 0));
    kern<<<grid, STEP_THREADS, 0, s>>>(H, a, wc);
}

template <bool CPLX, int G>
void launch_df_g(const SellView& H, StepMode mode, const StepArgs& a, int wc, int width, int sms,
                 cudaStream_t s) {
    switch (mode) {
        case MODE_SPMV: launch_df_gm<CPLX, G, MODE_SPMV>(H, a, wc, width, sms, s); break;
        case MODE_SECOND: launch_df_gm<CPLX, G, MODE_SECOND>(H, a, wc, width, sms, s); break;
        case MODE_STEP: launch_df_gm<CPLX, G, MODE_STEP>(H, a, wc, width, sms, s); break;
    }
}

template <bool CPLX>
void launch_df(const SellView& H, StepMode mode, const StepArgs& a, int wc, int width, int sms,
               cudaStream_t s) {
    if (wc > 16) launch_df_g<CPLX, 32>(H, mode, a, wc, width, sms, s);
    else if (wc > 8) launch_df_g<CPLX, 16>(H, mode, a, wc, width, sms, s);
    else if (wc > 4) launch_df_g<CPLX, 8>(H, mode, a, wc, width, sms, s);
    else launch_df_g<CPLX, 4>(H, mode, a, wc, width, sms, s);
}

}  // namespace chebfd
