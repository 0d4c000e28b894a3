// Double-float step kernels, complex values (see df_kernels.cuh).
#include "df_step.cuh"

namespace chebfd {

void launch_step_df_c(const SellView& H, StepMode mode, const StepArgs& a, int wc, int width,
                      int sms, cudaStream_t s) {
    launch_df<true>(H, mode, a, wc, width, sms, s);
}

}  // namespace chebfd
