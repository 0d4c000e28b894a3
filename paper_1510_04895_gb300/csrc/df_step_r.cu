// Double-float step kernels, real values (see df_kernels.cuh).
#include "df_step.cuh"

namespace chebfd {

void launch_step_df_r(const SellView& H, StepMode mode, const StepArgs& a, int wc, int width,
                      int sms, cudaStream_t s) {
    launch_df<false>(H, mode, a, wc, width, sms, s);
}

}  // namespace chebfd
