// The filter of Fig. ChebFD in double-float arithmetic on an FP64 block:
// each column panel is split into hi + lo floats, filtered with the
// double-float step kernels, and summed back into FP64.  This is the fast
// FP64-class sweep of the mixed-precision solve on GB300 (FP64 ALU ~1/64 of
// the FP32 rate; the double-float step runs on the paired FP32 pipe).
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "df.cuh"
#include "filter_kernels.cuh"

namespace chebfd {

void launch_step_df_c(const SellView& H, StepMode mode, const StepArgs& a, int wc, int width,
                      int sms, cudaStream_t s);
void launch_step_df_r(const SellView& H, StepMode mode, const StepArgs& a, int wc, int width,
                      int sms, cudaStream_t s);
void validate_block(const Matrix& M, chebfd_dtype dt, const void* X, int64_t ld, int nb);
bool stencil_df_applies(const Matrix& M, StepMode mode, int wc);
void launch_stencil_df(const Matrix& M, const StepArgs& a, int wc, cudaStream_t s);

namespace {

// Columns per panel: 32 complex or 64 real entries (32 chunks of 16 bytes).
int df_panel(bool cplx) { return cplx ? 32 : 64; }

// FP64 panel (cols [0, nb) of X, row stride ld entries) -> double-float chunks
// (row stride ldc): complex entry -> (re_hi, im_hi, re_lo, im_lo); real
// entries 2c, 2c+1 -> (x0_hi, x1_hi, x0_lo, x1_lo).
template <bool CPLX>
__global__ void to_df_kernel(const double* X, int64_t n, int64_t ld, int nb, float4* D,
                             int64_t ldc) {
    const int wc = CPLX ? nb : nb / 2;
    const int64_t total = n * wc;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / wc;
        const int c = (int)(t - i * wc);
        float h0, l0, h1, l1;
        if (CPLX) {
            df_split(X[2 * (i * ld + c)], h0, l0);
            df_split(X[2 * (i * ld + c) + 1], h1, l1);
        } else {
            df_split(X[i * ld + 2 * c], h0, l0);
            df_split(X[i * ld + 2 * c + 1], h1, l1);
        }
        D[i * ldc + c] = make_float4(h0, h1, l0, l1);
    }
}

template <bool CPLX>
__global__ void from_df_kernel(const float4* D, int64_t ldc, int64_t n, int nb, double* X,
                               int64_t ld) {
    const int wc = CPLX ? nb : nb / 2;
    const int64_t total = n * wc;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / wc;
        const int c = (int)(t - i * wc);
        const float4 d = D[i * ldc + c];
        const double v0 = (double)d.x + (double)d.z, v1 = (double)d.y + (double)d.w;
        if (CPLX) {
            X[2 * (i * ld + c)] = v0;
            X[2 * (i * ld + c) + 1] = v1;
        } else {
            X[i * ld + 2 * c] = v0;
            X[i * ld + 2 * c + 1] = v1;
        }
    }
}

int conv_grid(int64_t work) {
    return (int)std::min<int64_t>(std::max<int64_t>((work + 255) / 256, 1), 8192);
}

void launch_df(const Matrix& M, StepMode mode, const StepArgs& a, int wc, cudaStream_t s) {
    if (stencil_df_applies(M, mode, wc)) return launch_stencil_df(M, a, wc, s);
    SellView v;
    v.chunk_ptr = M.chunk_ptr;
    v.chunk_len = M.chunk_len;
    v.col = M.col;
    v.val = M.valdf;
    v.perm = M.identity_perm ? nullptr : M.perm;
    v.n = M.n;
    v.C = M.C;
    v.logC = 0;
    while ((1 << v.logC) < M.C) ++v.logC;
    StepArgs b = a;
    static const int env_tile = [] {
        const char* e = getenv("CHEBFD_STEP_TILE");
        return e ? std::max(1, atoi(e)) : 4;
    }();
    b.tile = env_tile;
    if (M.complex_values)
        launch_step_df_c(v, mode, b, wc, M.uniform_width, M.num_sms, s);
    else
        launch_step_df_r(v, mode, b, wc, M.uniform_width, M.num_sms, s);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

struct Buf {
    void* p = nullptr;
    cudaStream_t s;
    Buf(size_t bytes, cudaStream_t st) : s(st) {
        if (bytes) CHEBFD_CHECK_CUDA(cudaMallocAsync(&p, bytes, st));
    }
    ~Buf() {
        if (p) cudaFreeAsync(p, s);
    }
    Buf(const Buf&) = delete;
    Buf& operator=(const Buf&) = delete;
};

}  // namespace

void filter_block_df_impl(const Matrix& M, double alpha, double beta, const double* gc, int Np,
                          void* X, int64_t ld, int nb, cudaStream_t s) {
    const bool cplx = M.complex_values;
    const chebfd_dtype d64 = cplx ? CHEBFD_C128 : CHEBFD_R64;
    validate_block(M, d64, X, ld, nb);
    CHEBFD_REQUIRE(M.valdf != nullptr, CHEBFD_EINVAL,
                   "double-float filter needs a matrix built with also_single");
    CHEBFD_REQUIRE(gc != nullptr && Np >= 2, CHEBFD_EINVAL, "need Np >= 2 and coefficients");
    CHEBFD_REQUIRE(std::isfinite(alpha) && std::isfinite(beta), CHEBFD_EINVAL,
                   "alpha, beta must be finite");
    const int pw = df_panel(cplx);
    const int wmax = std::min(pw, nb);
    const int64_t ldc = cplx ? wmax : wmax / 2;  // chunks per row of the work panels
    const size_t bytes = (size_t)M.n * ldc * sizeof(float4);
    Buf D(bytes, s), U(bytes, s), W(bytes, s);
    for (int p0 = 0; p0 < nb; p0 += pw) {
        const int pnb = std::min(pw, nb - p0);
        const int wc = cplx ? pnb : pnb / 2;
        double* Xp = (double*)X + (cplx ? 2 : 1) * p0;
        if (cplx)
            to_df_kernel<true><<<conv_grid(M.n * wc), 256, 0, s>>>(Xp, M.n, ld, pnb, (float4*)D.p, ldc);
        else
            to_df_kernel<false><<<conv_grid(M.n * wc), 256, 0, s>>>(Xp, M.n, ld, pnb, (float4*)D.p, ldc);
        CHEBFD_CHECK_CUDA(cudaGetLastError());
        StepArgs a{};
        a.nb = pnb;
        a.alpha = alpha;
        a.beta = beta;
        a.ldg = a.ldw = a.ldy = ldc;
        // T_1 = A T_0 with T_0 = the panel D, into U
        a.gather = D.p;
        a.w = U.p;
        launch_df(M, MODE_SPMV, a, wc, s);
        // T_2 = 2 A T_1 - T_0 into W; D becomes gc_0 T_0 + gc_1 T_1 + gc_2 T_2
        a.gather = U.p;
        a.w = W.p;
        a.y = D.p;
        a.c0 = gc[0];
        a.c1 = gc[1];
        a.c2 = gc[2];
        launch_df(M, MODE_SECOND, a, wc, s);
        // n = 3..Np: T_n = 2 A T_{n-1} - T_{n-2} overwrites T_{n-2}; D gains gc_n T_n
        void* t_prev = U.p;
        void* t_cur = W.p;
        for (int k = 3; k <= Np; ++k) {
            a.gather = t_cur;
            a.w = t_prev;
            a.c0 = gc[k];
            launch_df(M, MODE_STEP, a, wc, s);
            std::swap(t_prev, t_cur);
        }
        if (cplx)
            from_df_kernel<true><<<conv_grid(M.n * wc), 256, 0, s>>>((const float4*)D.p, ldc, M.n, pnb, Xp, ld);
        else
            from_df_kernel<false><<<conv_grid(M.n * wc), 256, 0, s>>>((const float4*)D.p, ldc, M.n, pnb, Xp, ld);
        CHEBFD_CHECK_CUDA(cudaGetLastError());
    }
}

}  // namespace chebfd
