// Dense FP64 block operations of the ChebFD iteration (Sec. 3.1 steps 6-7):
// SVQB orthonormalisation, Rayleigh-Ritz projection, Ritz vectors and
// residual norms.  Tall-skinny products go to cuBLAS (FP64 GEMM/HERK), the
// small n_s x n_s Hermitian eigenproblems to cuSOLVER (FP64), everything else
// (scalings, symmetrisation, refill, residual norms, precision conversion) to
// the kernels below.
//
// A row-major N x n_s block Y is, for cuBLAS, the column-major n_s x N matrix
// Yc = Y^T.  Then cublas HERK/GEMM on Yc yield conj(Y^H Y) and conj(Y^H H Y);
// their eigenvectors are conj(U), and Y <- Y U becomes Yc <- U'^H Yc with
// U' = conj(U) - which is why the transforms below use CUBLAS_OP_C.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "common.cuh"

namespace chebfd {

void spmv_impl(const Matrix& M, double alpha, double beta, const void* X, void* Y, int64_t ld,
               int nb, chebfd_dtype dt, cudaStream_t s);
size_t df_gram_work_bytes(int m, int sms);
void df_gram(bool cplx, const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n,
             int m, double* C, void* work, int sms, cudaStream_t s);
void df_gemm(bool cplx, int r, int64_t n, int k, const double* Mt, int ldm, const double* Y,
             int64_t ldy, double* T, int64_t ldt, cudaStream_t s);
void oz_gram(bool cplx, const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n,
             int m, double* C, int sms, cudaStream_t s);
void check_oz_errors(cudaStream_t s);
void oz_gemm(bool cplx, int r, int64_t n, int k, const double* M, int ldm, const double* Y,
             int64_t ldy, double* T, int64_t ldt, int sms, cudaStream_t s, bool conj);
void oz_gram_rect(bool cplx, const double* A, int64_t lda, int ma, const double* B, int64_t ldb,
                  int mb, int64_t n, double* C, int sms, cudaStream_t s);

namespace {

#define CHEBFD_CHECK_CUBLAS(expr)                                                         \
    do {                                                                                  \
        cublasStatus_t st_ = (expr);                                                      \
        if (st_ != CUBLAS_STATUS_SUCCESS)                                                 \
            throw ::chebfd::Error{st_ == CUBLAS_STATUS_ALLOC_FAILED ? CHEBFD_ENOMEM        \
                                                                    : CHEBFD_ECUDA,       \
                                  std::string(#expr) + " failed: " + std::to_string(st_)}; \
    } while (0)
#define CHEBFD_CHECK_CUSOLVER(expr)                                                       \
    do {                                                                                  \
        cusolverStatus_t st_ = (expr);                                                    \
        if (st_ != CUSOLVER_STATUS_SUCCESS)                                               \
            throw ::chebfd::Error{CHEBFD_ECUDA,                                           \
                                  std::string(#expr) + " failed: " + std::to_string(st_)}; \
    } while (0)

struct Handles {
    cublasHandle_t blas = nullptr;
    cusolverDnHandle_t solver = nullptr;
};

// One cuBLAS / cuSOLVER handle pair per host thread and device: a handle is
// bound to one stream at a time, so threads never share one.  The handles
// live until the process exits.
Handles& handles_for_current_device(cudaStream_t s) {
    thread_local std::map<int, Handles> cache;
    int dev = 0;
    CHEBFD_CHECK_CUDA(cudaGetDevice(&dev));
    Handles& h = cache[dev];
    if (!h.blas) CHEBFD_CHECK_CUBLAS(cublasCreate(&h.blas));
    if (!h.solver) CHEBFD_CHECK_CUSOLVER(cusolverDnCreate(&h.solver));
    CHEBFD_CHECK_CUBLAS(cublasSetStream(h.blas, s));
    CHEBFD_CHECK_CUBLAS(cublasSetPointerMode(h.blas, CUBLAS_POINTER_MODE_HOST));
    CHEBFD_CHECK_CUSOLVER(cusolverDnSetStream(h.solver, s));
    return h;
}

struct Buf {
    void* p = nullptr;
    cudaStream_t s;
    Buf(size_t bytes, cudaStream_t st) : s(st) {
        if (bytes) CHEBFD_CHECK_CUDA(cudaMallocAsync(&p, bytes, st));
    }
    ~Buf() { reset(); }
    void reset() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
    }
    Buf(const Buf&) = delete;
    Buf& operator=(const Buf&) = delete;
    template <class T>
    T* as() const {
        return reinterpret_cast<T*>(p);
    }
};

int grid1d(int64_t work) {
    return (int)std::min<int64_t>(std::max<int64_t>((work + 255) / 256, 1), 8192);
}

// ----------------------------------------------------------------- small kernels

// d_i = Re(S_ii)^(-1/2) (0 for a zero column); S <- D S D.  One block: the
// diagonal is read before any element is scaled.
template <bool CPLX>
__global__ void diag_scale_kernel(double* S, int ns, double* d) {
    __shared__ double dd[1024];
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        const double sii = CPLX ? S[2 * ((int64_t)i * ns + i)] : S[(int64_t)i * ns + i];
        const double v = sii > 0.0 ? 1.0 / sqrt(sii) : 0.0;
        dd[i] = v;
        d[i] = v;
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < (int64_t)ns * ns; t += blockDim.x) {
        const int col = (int)(t / ns), row = (int)(t % ns);  // column-major
        const double f = dd[row] * dd[col];
        if (CPLX) {
            S[2 * t] *= f;
            S[2 * t + 1] *= f;
        } else {
            S[t] *= f;
        }
    }
}

// M'[:, j] = D U'[:, first + j] Theta_{first+j}^(-1/2), j < r (column-major ns x r).
template <bool CPLX>
__global__ void form_transform_kernel(const double* U, const double* d, const double* theta,
                                      int ns, int first, int r, double* Mt) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)ns * r;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / ns), i = (int)(t % ns);
        const double f = d[i] / sqrt(theta[first + j]);
        const int64_t src = (int64_t)(first + j) * ns + i;
        if (CPLX) {
            Mt[2 * t] = U[2 * src] * f;
            Mt[2 * t + 1] = U[2 * src + 1] * f;
        } else {
            Mt[t] = U[src] * f;
        }
    }
}

// G <- (G + G^H) / 2 for a full column-major ns x ns matrix.
template <bool CPLX>
__global__ void hermitize_kernel(double* G, int ns) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)ns * ns;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / ns), r = (int)(t % ns);
        if (r < c) continue;
        const int64_t u = (int64_t)r * ns + c;  // element (c, r)
        if (CPLX) {
            const double re = 0.5 * (G[2 * t] + G[2 * u]);
            const double im = 0.5 * (G[2 * t + 1] - G[2 * u + 1]);
            G[2 * t] = re;
            G[2 * t + 1] = im;
            G[2 * u] = re;
            G[2 * u + 1] = -im;
        } else {
            const double v = 0.5 * (G[t] + G[u]);
            G[t] = v;
            G[u] = v;
        }
    }
}

// max |S - I| over the lower triangle of a column-major ns x ns matrix: one block.
template <bool CPLX>
__global__ void max_offidentity_kernel(const double* S, int ns, double* out) {
    __shared__ double m[256];
    double v = 0.0;
    for (int64_t t = threadIdx.x; t < (int64_t)ns * ns; t += blockDim.x) {
        const int c = (int)(t / ns), r = (int)(t % ns);
        if (r < c) continue;
        double re = CPLX ? S[2 * t] : S[t];
        const double im = CPLX ? S[2 * t + 1] : 0.0;
        if (r == c) re -= 1.0;
        v = fmax(v, sqrt(re * re + im * im));
    }
    m[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) m[threadIdx.x] = fmax(m[threadIdx.x], m[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = m[0];
}

// Refill columns [c0, ns) of a row-major block with random vectors of stream 3:
// the q-th refill column of the run (q = counter + k - c0) has entries 2u - 1 at
// word indices q*N + i (real) or 2(q*N + i) + {0, 1} (complex).
template <bool CPLX>
__global__ void refill_kernel(double* Y, int64_t n, int64_t ld, int c0, int ns, int64_t counter,
                              uint64_t seed) {
    const int w = ns - c0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * w;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / w;
        const int k = c0 + (int)(t - i * w);
        const uint64_t q = (uint64_t)(counter + k - c0);
        if (CPLX) {
            const uint64_t idx = 2 * (q * (uint64_t)n + (uint64_t)i);
            Y[2 * (i * ld + k)] = 2.0 * splitmix_uniform(seed, STREAM_REFILL, idx) - 1.0;
            Y[2 * (i * ld + k) + 1] = 2.0 * splitmix_uniform(seed, STREAM_REFILL, idx + 1) - 1.0;
        } else {
            Y[i * ld + k] =
                2.0 * splitmix_uniform(seed, STREAM_REFILL, q * (uint64_t)n + (uint64_t)i) - 1.0;
        }
    }
}

// Per-column partial sums of |HV_ik - theta_k V_ik|^2 over a row range; one
// partial per block, summed later in block order.
template <bool CPLX>
__global__ void residual_partials_kernel(const double* HV, const double* V, const double* theta,
                                         int64_t n, int64_t ld, int k, double* part) {
    const int64_t rows_per_block = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * rows_per_block;
    const int64_t r1 = min(n, r0 + rows_per_block);
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        const double th = theta[c];
        double acc = 0.0;
        for (int64_t i = r0; i < r1; ++i) {
            if (CPLX) {
                const double dr = HV[2 * (i * ld + c)] - th * V[2 * (i * ld + c)];
                const double di = HV[2 * (i * ld + c) + 1] - th * V[2 * (i * ld + c) + 1];
                acc += dr * dr + di * di;
            } else {
                const double dr = HV[i * ld + c] - th * V[i * ld + c];
                acc += dr * dr;
            }
        }
        part[(int64_t)blockIdx.x * k + c] = acc;
    }
}

__global__ void sum_partials_kernel(const double* part, int blocks, int k, double* out) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < k; c += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < blocks; ++b) s += part[(int64_t)b * k + c];
        out[c] = sqrt(s);
    }
}

template <class From, class To>
__global__ void convert_kernel(const From* x, int64_t ldx, To* y, int64_t ldy, int64_t n,
                               int w) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * w;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / w;
        const int k = (int)(t - i * w);
        y[i * ldy + k] = (To)x[i * ldx + k];
    }
}

// ----------------------------------------------------------------- BLAS wrappers

// Cc (m x m) = A (m x n) * B^H (n x m).
void gemm_nh(Handles& h, bool cplx, int m, int64_t n, const double* A, int64_t lda,
             const double* B, int64_t ldb, double* Cc, int ldc);

// conj(Y^H Y) (column-major ns x ns, full) through GEMM: for tall blocks
// (N >> ns) the library's GEMM splits the long dimension across the GPU,
// where the rank-k update (HERK) measured ~3x slower on GB300.
void gram(Handles& h, bool cplx, const double* Y, int64_t n, int ns, int64_t ld, double* S) {
    gemm_nh(h, cplx, ns, n, Y, ld, Y, ld, S, ns);
}

// Cc (m x n, ldc) = op(A) (m x k) * B (k x n), op = conjugate transpose.
void gemm_ch(Handles& h, bool cplx, int m, int64_t n, int k, const double* A, int lda,
             const double* B, int64_t ldb, double* Cc, int64_t ldc) {
    if (cplx) {
        const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0),
                              zero = make_cuDoubleComplex(0.0, 0.0);
        CHEBFD_CHECK_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_C, CUBLAS_OP_N, m, (int)n, k, &one,
                                        (const cuDoubleComplex*)A, lda,
                                        (const cuDoubleComplex*)B, (int)ldb, &zero,
                                        (cuDoubleComplex*)Cc, (int)ldc));
    } else {
        const double one = 1.0, zero = 0.0;
        CHEBFD_CHECK_CUBLAS(cublasDgemm(h.blas, CUBLAS_OP_T, CUBLAS_OP_N, m, (int)n, k, &one, A,
                                        lda, B, (int)ldb, &zero, Cc, (int)ldc));
    }
}

// Cc (m x m) = A (m x n) * B^H (n x m).
void gemm_nh(Handles& h, bool cplx, int m, int64_t n, const double* A, int64_t lda,
             const double* B, int64_t ldb, double* Cc, int ldc) {
    if (cplx) {
        const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0),
                              zero = make_cuDoubleComplex(0.0, 0.0);
        CHEBFD_CHECK_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_C, m, m, (int)n, &one,
                                        (const cuDoubleComplex*)A, (int)lda,
                                        (const cuDoubleComplex*)B, (int)ldb, &zero,
                                        (cuDoubleComplex*)Cc, ldc));
    } else {
        const double one = 1.0, zero = 0.0;
        CHEBFD_CHECK_CUBLAS(cublasDgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_T, m, m, (int)n, &one, A,
                                        (int)lda, B, (int)ldb, &zero, Cc, ldc));
    }
}

// Hermitian eigensolve of the lower triangle of A (ns x ns, in place: vectors).
void heev(Handles& h, bool cplx, double* A, int ns, double* w, cudaStream_t s) {
    int lwork = 0;
    if (cplx)
        CHEBFD_CHECK_CUSOLVER(cusolverDnZheevd_bufferSize(
            h.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, ns,
            (cuDoubleComplex*)A, ns, w, &lwork));
    else
        CHEBFD_CHECK_CUSOLVER(cusolverDnDsyevd_bufferSize(h.solver, CUSOLVER_EIG_MODE_VECTOR,
                                                          CUBLAS_FILL_MODE_LOWER, ns, A, ns, w,
                                                          &lwork));
    Buf work((size_t)std::max(lwork, 1) * (cplx ? 16 : 8), s);
    Buf info(sizeof(int), s);
    if (cplx)
        CHEBFD_CHECK_CUSOLVER(cusolverDnZheevd(h.solver, CUSOLVER_EIG_MODE_VECTOR,
                                               CUBLAS_FILL_MODE_LOWER, ns, (cuDoubleComplex*)A,
                                               ns, w, work.as<cuDoubleComplex>(), lwork,
                                               info.as<int>()));
    else
        CHEBFD_CHECK_CUSOLVER(cusolverDnDsyevd(h.solver, CUSOLVER_EIG_MODE_VECTOR,
                                               CUBLAS_FILL_MODE_LOWER, ns, A, ns, w,
                                               work.as<double>(), lwork, info.as<int>()));
    int hinfo = 0;
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
    CHEBFD_REQUIRE(hinfo == 0, CHEBFD_ENUMERIC, "dense eigensolver did not converge");
}

// Hermitian-definite generalized eigensolve A x = mu B x (lower triangles;
// A <- vectors normalised to x^H B x = 1, B <- its Cholesky factor, mu
// ascending).  Returns false when B is not positive definite.
bool hegv(Handles& h, bool cplx, double* A, double* B, int ns, double* w, cudaStream_t s) {
    int lwork = 0;
    if (cplx)
        CHEBFD_CHECK_CUSOLVER(cusolverDnZhegvd_bufferSize(
            h.solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, ns,
            (cuDoubleComplex*)A, ns, (cuDoubleComplex*)B, ns, w, &lwork));
    else
        CHEBFD_CHECK_CUSOLVER(cusolverDnDsygvd_bufferSize(
            h.solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, ns,
            A, ns, B, ns, w, &lwork));
    Buf work((size_t)std::max(lwork, 1) * (cplx ? 16 : 8), s);
    Buf info(sizeof(int), s);
    if (cplx)
        CHEBFD_CHECK_CUSOLVER(cusolverDnZhegvd(
            h.solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, ns,
            (cuDoubleComplex*)A, ns, (cuDoubleComplex*)B, ns, w, work.as<cuDoubleComplex>(),
            lwork, info.as<int>()));
    else
        CHEBFD_CHECK_CUSOLVER(cusolverDnDsygvd(
            h.solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, ns, A,
            ns, B, ns, w, work.as<double>(), lwork, info.as<int>()));
    int hinfo = 0;
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
    if (hinfo > ns) return false;  // leading minor of B not positive definite
    CHEBFD_REQUIRE(hinfo == 0, CHEBFD_ENUMERIC, "generalized eigensolver did not converge");
    return true;
}

void copy_block(void* dst, int64_t ldd, const void* src, int64_t lds, int64_t n, int w,
                size_t es, cudaStream_t s) {
    CHEBFD_CHECK_CUDA(cudaMemcpy2DAsync(dst, ldd * es, src, lds * es, (size_t)w * es, n,
                                        cudaMemcpyDeviceToDevice, s));
}

void check_fp64_block(chebfd_dtype dt, const void* Y, int64_t n, int ns, int64_t ld) {
    CHEBFD_REQUIRE(dt == CHEBFD_R64 || dt == CHEBFD_C128, CHEBFD_EINVAL,
                   "dense steps run in FP64: dtype must be R64 or C128");
    CHEBFD_REQUIRE(Y != nullptr && n >= 1 && ns >= 1 && ld >= ns, CHEBFD_EINVAL,
                   "bad block arguments");
    CHEBFD_REQUIRE(ns <= 1024, CHEBFD_EINVAL, "n_s > 1024 is not supported");
    CHEBFD_REQUIRE(n < (1LL << 31), CHEBFD_EINVAL, "N must be < 2^31");
    CHEBFD_REQUIRE((uintptr_t)Y % 16 == 0, CHEBFD_EINVAL, "block must be 16-byte aligned");
}

}  // namespace

void residuals_from_blocks(bool cplx, const double* HV, const double* V, const double* theta_dev,
                           int64_t n, int64_t ld, int k, double* res_dev, cudaStream_t s) {
    const int blocks = (int)std::min<int64_t>(1024, std::max<int64_t>(1, n / 64));
    Buf part((size_t)blocks * k * sizeof(double), s);
    if (cplx)
        residual_partials_kernel<true><<<blocks, 256, 0, s>>>(HV, V, theta_dev, n, ld, k,
                                                              part.as<double>());
    else
        residual_partials_kernel<false><<<blocks, 256, 0, s>>>(HV, V, theta_dev, n, ld, k,
                                                               part.as<double>());
    sum_partials_kernel<<<(k + 255) / 256, 256, 0, s>>>(part.as<double>(), blocks, k, res_dev);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

namespace {

// Y[i][k] -= T[i][k] for k < w doubles per row (Y: ld, T: ldt doubles per row).
__global__ void sub_block_kernel(double* __restrict__ Y, int64_t ld, const double* __restrict__ T,
                                 int64_t ldt, int64_t n, int w) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * w;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / w;
        const int k = (int)(t - i * w);
        Y[i * ld + k] -= T[i * ldt + k];
    }
}

// dst[i][j] = src[i][idx[j]] (entries of ew doubles), j < cnt.
__global__ void gather_columns_kernel(const double* __restrict__ src, int64_t ld, int64_t n,
                                      const int* __restrict__ idx, int cnt, int ew,
                                      double* __restrict__ dst, int64_t ldd) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * cnt;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / cnt;
        const int j = (int)(t - i * cnt);
        for (int e = 0; e < ew; ++e) dst[(i * ldd + j) * ew + e] = src[(i * ld + idx[j]) * ew + e];
    }
}

}  // namespace

// Y (N x w, ld) <- Y - L (L^H Y), twice, for the locked vectors L (N x nl,
// ld): the rectangular Gram and block product on the tensor cores (tensor)
// or with cuBLAS FP64.  Hard locking of converged pairs (Sec. 6).
void deflate_impl(bool cplx, const double* L, int nl, double* Y, int w, int64_t n, int64_t ld,
                  bool tensor, int sms, cudaStream_t s) {
    if (nl <= 0 || w <= 0) return;
    const size_t es = cplx ? 16 : 8;
    Buf C((size_t)nl * w * es, s), T((size_t)n * w * es, s);
    Handles& h = handles_for_current_device(s);
    for (int pass = 0; pass < 2; ++pass) {
        // C[p + q nl] = sum_i L[i,p] conj(Y[i,q]);  T = L conj(C) = L (L^H Y)
        if (tensor) {
            oz_gram_rect(cplx, L, ld, nl, Y, ld, w, n, C.as<double>(), sms, s);
            oz_gemm(cplx, w, n, nl, C.as<double>(), nl, L, ld, T.as<double>(), w, sms, s, true);
        } else {
            if (cplx) {
                const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0),
                                      zero = make_cuDoubleComplex(0.0, 0.0);
                CHEBFD_CHECK_CUBLAS(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_C, nl, w, (int)n,
                                                &one, (const cuDoubleComplex*)L, (int)ld,
                                                (const cuDoubleComplex*)Y, (int)ld, &zero,
                                                C.as<cuDoubleComplex>(), nl));
            } else {
                const double one = 1.0, zero = 0.0;
                CHEBFD_CHECK_CUBLAS(cublasDgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_T, nl, w, (int)n,
                                                &one, L, (int)ld, Y, (int)ld, &zero,
                                                C.as<double>(), nl));
            }
            gemm_ch(h, cplx, w, n, nl, C.as<double>(), nl, L, ld, T.as<double>(), w);
        }
        const int ew = cplx ? 2 : 1;
        sub_block_kernel<<<grid1d(n * w * ew), 256, 0, s>>>(Y, ld * ew, T.as<double>(), (int64_t)w * ew,
                                                            n, w * ew);
        CHEBFD_CHECK_CUDA(cudaGetLastError());
    }
}

// dst[i][j] = src[i][idx[j]] for FP64 blocks (complex: 2 doubles per entry).
void gather_columns_impl(const double* src, int64_t ld, int64_t n, const std::vector<int>& idx,
                         bool cplx, double* dst, int64_t ldd, cudaStream_t s) {
    if (idx.empty()) return;
    Buf d((size_t)idx.size() * sizeof(int), s);
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(d.p, idx.data(), idx.size() * sizeof(int),
                                      cudaMemcpyHostToDevice, s));
    gather_columns_kernel<<<grid1d(n * (int64_t)idx.size()), 256, 0, s>>>(
        src, ld, n, d.as<int>(), (int)idx.size(), cplx ? 2 : 1, dst, ldd);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));   // idx buffer freed after the copy
}

void orthonormalize_impl(void* Yv, int64_t n, int ns, int64_t ld, chebfd_dtype dt,
                         uint64_t seed, int64_t* refill_counter, int* rank_out, cudaStream_t s) {
    check_fp64_block(dt, Yv, n, ns, ld);
    const bool cplx = dt == CHEBFD_C128;
    const size_t es = cplx ? 16 : 8;
    double* Y = (double*)Yv;
    Handles& h = handles_for_current_device(s);
    Buf S((size_t)ns * ns * es, s), d((size_t)ns * sizeof(double), s),
        th((size_t)ns * sizeof(double), s), Mt((size_t)ns * ns * es, s),
        T((size_t)n * ld * es, s), err(sizeof(double), s);
    std::vector<double> hth(ns);
    int64_t counter = refill_counter ? *refill_counter : 0;
    int first_rank = -1;
    gram(h, cplx, Y, n, ns, ld, S.as<double>());
    for (int pass = 0; pass < 3; ++pass) {
        if (cplx)
            diag_scale_kernel<true><<<1, 1024, 0, s>>>(S.as<double>(), ns,
                                                                             d.as<double>());
        else
            diag_scale_kernel<false><<<1, 1024, 0, s>>>(S.as<double>(), ns,
                                                                              d.as<double>());
        heev(h, cplx, S.as<double>(), ns, th.as<double>(), s);
        CHEBFD_CHECK_CUDA(cudaMemcpyAsync(hth.data(), th.p, ns * sizeof(double),
                                          cudaMemcpyDeviceToHost, s));
        CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
        const double thr = ns * std::ldexp(1.0, -52) * hth[ns - 1];
        int first = 0;
        while (first < ns && !(hth[first] >= thr)) ++first;
        const int r = ns - first;
        CHEBFD_REQUIRE(r >= 1, CHEBFD_ENUMERIC, "orthonormalisation: block has rank 0");
        if (first_rank < 0) first_rank = r;
        if (cplx)
            form_transform_kernel<true><<<grid1d((int64_t)ns * r), 256, 0, s>>>(
                S.as<double>(), d.as<double>(), th.as<double>(), ns, first, r, Mt.as<double>());
        else
            form_transform_kernel<false><<<grid1d((int64_t)ns * r), 256, 0, s>>>(
                S.as<double>(), d.as<double>(), th.as<double>(), ns, first, r, Mt.as<double>());
        // T (row-major, first r columns) = Y M
        gemm_ch(h, cplx, r, n, ns, Mt.as<double>(), ns, Y, ld, T.as<double>(), ld);
        if (r < ns) {
            if (cplx)
                refill_kernel<true><<<grid1d(n * (ns - r)), 256, 0, s>>>(T.as<double>(), n, ld, r,
                                                                         ns, counter, seed);
            else
                refill_kernel<false><<<grid1d(n * (ns - r)), 256, 0, s>>>(T.as<double>(), n, ld,
                                                                          r, ns, counter, seed);
            counter += ns - r;
        }
        copy_block(Y, ld, T.p, ld, n, ns, es, s);
        gram(h, cplx, Y, n, ns, ld, S.as<double>());
        if (r < ns) continue;
        if (cplx)
            max_offidentity_kernel<true><<<1, 256, 0, s>>>(S.as<double>(), ns, err.as<double>());
        else
            max_offidentity_kernel<false><<<1, 256, 0, s>>>(S.as<double>(), ns, err.as<double>());
        double herr = 0.0;
        CHEBFD_CHECK_CUDA(
            cudaMemcpyAsync(&herr, err.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
        if (herr <= 1e-12) break;
    }
    CHEBFD_CHECK_CUDA(cudaGetLastError());
    if (refill_counter) *refill_counter = counter;
    if (rank_out) *rank_out = first_rank;
}

// Rayleigh-Ritz of Sec. 3.1 step 7 on an orthonormal FP64 block Y (in place:
// Y <- Ritz vectors, ascending theta).  theta_host/res_host: ns doubles (res
// may be null).  HY_out (nullable, N x ns, ld) receives H V.
void rayleigh_ritz_impl(const Matrix& M, void* Yv, int64_t ld, int ns, chebfd_dtype dt,
                        double* theta_host, double* res_host, void* HY_out, cudaStream_t s) {
    check_fp64_block(dt, Yv, M.n, ns, ld);
    CHEBFD_REQUIRE(theta_host != nullptr, CHEBFD_EINVAL, "null theta");
    const bool cplx = dt == CHEBFD_C128;
    CHEBFD_REQUIRE(cplx == M.complex_values, CHEBFD_EINVAL, "dtype does not match the matrix");
    const size_t es = cplx ? 16 : 8;
    const int64_t n = M.n;
    double* Y = (double*)Yv;
    Handles& h = handles_for_current_device(s);
    Buf HY((size_t)n * ld * es, s), T((size_t)n * ld * es, s), G((size_t)ns * ns * es, s),
        th((size_t)ns * sizeof(double), s), res((size_t)ns * sizeof(double), s);
    // H Y through the fused kernel in plain-product mode
    spmv_impl(M, 1.0, 0.0, Y, HY.p, ld, ns, dt, s);
    // G^T = conj(Y^H H Y) (column-major), made exactly Hermitian
    gemm_nh(h, cplx, ns, n, HY.as<double>(), ld, Y, ld, G.as<double>(), ns);
    if (cplx)
        hermitize_kernel<true><<<grid1d((int64_t)ns * ns), 256, 0, s>>>(G.as<double>(), ns);
    else
        hermitize_kernel<false><<<grid1d((int64_t)ns * ns), 256, 0, s>>>(G.as<double>(), ns);
    heev(h, cplx, G.as<double>(), ns, th.as<double>(), s);
    // V = Y S, HV = HY S  (Vc = S'^H Yc)
    gemm_ch(h, cplx, ns, n, ns, G.as<double>(), ns, Y, ld, T.as<double>(), ld);
    copy_block(Y, ld, T.p, ld, n, ns, es, s);
    gemm_ch(h, cplx, ns, n, ns, G.as<double>(), ns, HY.as<double>(), ld, T.as<double>(), ld);
    residuals_from_blocks(cplx, T.as<double>(), Y, th.as<double>(), n, ld, ns, res.as<double>(), s);
    if (HY_out) copy_block(HY_out, ld, T.p, ld, n, ns, es, s);
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(theta_host, th.p, ns * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
    if (res_host)
        CHEBFD_CHECK_CUDA(cudaMemcpyAsync(res_host, res.p, ns * sizeof(double),
                                          cudaMemcpyDeviceToHost, s));
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
}

namespace {

// C (ns x ns, column-major) = op(A) * B, op = conjugate transpose if ah.
void gemm_small(Handles& h, bool cplx, bool ah, int ns, const double* A, const double* B,
                double* C) {
    if (cplx) {
        const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0),
                              zero = make_cuDoubleComplex(0.0, 0.0);
        CHEBFD_CHECK_CUBLAS(cublasZgemm(h.blas, ah ? CUBLAS_OP_C : CUBLAS_OP_N, CUBLAS_OP_N, ns,
                                        ns, ns, &one, (const cuDoubleComplex*)A, ns,
                                        (const cuDoubleComplex*)B, ns, &zero,
                                        (cuDoubleComplex*)C, ns));
    } else {
        const double one = 1.0, zero = 0.0;
        CHEBFD_CHECK_CUBLAS(cublasDgemm(h.blas, ah ? CUBLAS_OP_T : CUBLAS_OP_N, CUBLAS_OP_N, ns,
                                        ns, ns, &one, A, ns, B, ns, &zero, C, ns));
    }
}

}  // namespace

// Harmonic Ritz extraction (the alternative to step 7 named in Sec. 3.1 and
// Sec. 6; Morgan 1991, Paige-Parlett-van der Vorst 1995) on an orthonormal
// FP64 block Y, target tau.  Z = (H - tau) Y through the fused kernel;
// A = Y^H Z and K = Z^H Z (stored conjugated, like every small matrix here);
// A s = mu K s with K positive definite gives the harmonic values tau + 1/mu.
// Each harmonic vector v = Y s / ||s|| gets its Rayleigh quotient
// rho = tau + mu / ||s||^2 (s^H A s = mu for K-normalised s) and the residual
// ||Z s - (rho - tau) Y s|| / ||s|| = ||H v - rho v||.  In place: Y <- unit
// harmonic vectors, ascending rho; theta_host <- rho.  When K is singular (a
// column of Y is an exact eigenvector at tau) this falls back to the Ritz
// pairs of A + tau.  tall_gram(X, W, C): C = conj(W^H X); tall_gemm(r, E, X, T):
// T = X conj(E).
template <class Gram, class Gemm>
void harmonic_extract(const Matrix& M, double* Y, int64_t ld, int ns, bool cplx, double tau,
                      Handles& h, Gram&& tall_gram, Gemm&& tall_gemm, double* theta_host,
                      double* res_host, cudaStream_t s, PhaseClock* clk = nullptr) {
    auto mark = [&](int ph) {
        if (clk) clk->mark(ph);
    };
    const size_t es = cplx ? 16 : 8;
    const int64_t n = M.n;
    const int ew = cplx ? 2 : 1;  // doubles per entry
    Buf Z((size_t)n * ld * es, s), T((size_t)n * ld * es, s), A((size_t)ns * ns * es, s),
        A0((size_t)ns * ns * es, s), K((size_t)ns * ns * es, s), w((size_t)ns * sizeof(double), s),
        dth((size_t)ns * sizeof(double), s), res((size_t)ns * sizeof(double), s);
    spmv_impl(M, 1.0, -tau, Y, Z.p, ld, ns, cplx ? CHEBFD_C128 : CHEBFD_R64, s);
    mark(PH_HY);
    tall_gram(Z.as<double>(), Y, A.as<double>());
    tall_gram(Z.as<double>(), Z.as<double>(), K.as<double>());
    mark(PH_GRAM);
    if (cplx) {
        hermitize_kernel<true><<<grid1d((int64_t)ns * ns), 256, 0, s>>>(A.as<double>(), ns);
        hermitize_kernel<true><<<grid1d((int64_t)ns * ns), 256, 0, s>>>(K.as<double>(), ns);
    } else {
        hermitize_kernel<false><<<grid1d((int64_t)ns * ns), 256, 0, s>>>(A.as<double>(), ns);
        hermitize_kernel<false><<<grid1d((int64_t)ns * ns), 256, 0, s>>>(K.as<double>(), ns);
    }
    CHEBFD_CHECK_CUDA(cudaGetLastError());
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(A0.p, A.p, (size_t)ns * ns * es, cudaMemcpyDeviceToDevice, s));
    std::vector<double> hw(ns), E((size_t)ns * ns * ew), nrm(ns, 1.0), rho(ns);
    const bool definite = hegv(h, cplx, A.as<double>(), K.as<double>(), ns, w.as<double>(), s);
    double* Ev = A.as<double>();
    if (!definite) {
        // Ritz pairs of A + tau = Y^H H Y instead
        CHEBFD_CHECK_CUDA(cudaMemcpyAsync(E.data(), A0.p, (size_t)ns * ns * es,
                                          cudaMemcpyDeviceToHost, s));
        CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < ns; ++i) E[(size_t)ew * ((size_t)i * ns + i)] += tau;
        CHEBFD_CHECK_CUDA(cudaMemcpyAsync(A0.p, E.data(), (size_t)ns * ns * es,
                                          cudaMemcpyHostToDevice, s));
        heev(h, cplx, A0.as<double>(), ns, w.as<double>(), s);
        Ev = A0.as<double>();
    }
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(hw.data(), w.p, ns * sizeof(double), cudaMemcpyDeviceToHost, s));
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(E.data(), Ev, (size_t)ns * ns * es, cudaMemcpyDeviceToHost, s));
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < ns; ++k) {
        if (definite) {
            double q = 0.0;
            for (int i = 0; i < ns * ew; ++i) q += E[(size_t)k * ns * ew + i] * E[(size_t)k * ns * ew + i];
            nrm[k] = std::sqrt(q);
            rho[k] = tau + hw[k] / q;
        } else {
            rho[k] = hw[k];
        }
    }
    std::vector<int> order(ns);
    for (int k = 0; k < ns; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return rho[x] < rho[y]; });
    std::vector<double> En((size_t)ns * ns * ew), dh(ns);
    for (int j = 0; j < ns; ++j) {
        const int k = order[j];
        const double f = nrm[k] > 0.0 ? 1.0 / nrm[k] : 0.0;
        for (int i = 0; i < ns * ew; ++i)
            En[(size_t)j * ns * ew + i] = E[(size_t)k * ns * ew + i] * f;
        theta_host[j] = rho[k];
        dh[j] = rho[k] - tau;
    }
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(A.p, En.data(), (size_t)ns * ns * es, cudaMemcpyHostToDevice, s));
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(dth.p, dh.data(), ns * sizeof(double), cudaMemcpyHostToDevice, s));
    mark(PH_EIG);
    // V = Y conj(En) into T, Z conj(En) into Y, residuals, Y <- V
    tall_gemm(ns, A.as<double>(), Y, T.as<double>());
    tall_gemm(ns, A.as<double>(), Z.as<double>(), Y);
    mark(PH_BLOCK_GEMM);
    residuals_from_blocks(cplx, Y, T.as<double>(), dth.as<double>(), n, ld, ns, res.as<double>(), s);
    copy_block(Y, ld, T.p, ld, n, ns, es, s);
    if (res_host)
        CHEBFD_CHECK_CUDA(cudaMemcpyAsync(res_host, res.p, ns * sizeof(double),
                                          cudaMemcpyDeviceToHost, s));
    mark(PH_RESIDUAL);
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

void harmonic_ritz_impl(const Matrix& M, void* Yv, int64_t ld, int ns, chebfd_dtype dt, double tau,
                        double* theta_host, double* res_host, cudaStream_t s) {
    check_fp64_block(dt, Yv, M.n, ns, ld);
    CHEBFD_REQUIRE(theta_host != nullptr, CHEBFD_EINVAL, "null theta");
    CHEBFD_REQUIRE(std::isfinite(tau), CHEBFD_EINVAL, "tau must be finite");
    const bool cplx = dt == CHEBFD_C128;
    CHEBFD_REQUIRE(cplx == M.complex_values, CHEBFD_EINVAL, "dtype does not match the matrix");
    const int64_t n = M.n;
    Handles& h = handles_for_current_device(s);
    auto gram_blas = [&](const double* X, const double* W, double* C) {
        gemm_nh(h, cplx, ns, n, X, ld, W, ld, C, ns);
    };
    auto gemm_blas = [&](int r, const double* E, const double* X, double* T) {
        gemm_ch(h, cplx, r, n, ns, E, ns, X, ld, T, ld);
    };
    harmonic_extract(M, (double*)Yv, ld, ns, cplx, tau, h, gram_blas, gemm_blas, theta_host,
                     res_host, s);
}

// Steps 6-7 of Sec. 3.1 in one pass over the dense work: two SVQB passes and
// the Rayleigh-Ritz projection, with the second SVQB transform folded into
// the projection instead of applied to the block.  With Y1 = Y T1 (pass 1,
// refill as in orthonormalize_impl), the second transform T2 comes from
// Y1^H Y1, and Y2 = Y1 T2 is never formed: Y2^H H Y2 = T2^H (Y1^H H Y1) T2 is
// an n_s x n_s product, and the Ritz vectors and their products with H are
// V = Y1 (T2 S), HV = (H Y1)(T2 S).  Tall products: three Gram-type GEMMs
// (Y^H Y, Y1^H Y1, Y1^H H Y1) and three block GEMMs (Y T1, V, HV) instead of
// the five + three of the separate calls.  A rank drop in the second pass
// falls back to the separate calls.  Y <- Ritz vectors (ascending theta).
// df: the six tall products in double-float arithmetic (df_dense.cu) instead
// of cuBLAS FP64; the n_s x n_s steps stay FP64.
// harmonic: harmonic Ritz pairs for the target tau (harmonic_extract) in the
// orthonormal basis Y2 = Y1 T2, formed explicitly, instead of Ritz pairs.
void ortho_rr_impl(const Matrix& M, void* Yv, int64_t ld, int ns, chebfd_dtype dt, uint64_t seed,
                   int64_t* refill_counter, double* theta_host, double* res_host, bool df,
                   bool harmonic, double tau, cudaStream_t s, double* phase_seconds) {
    check_fp64_block(dt, Yv, M.n, ns, ld);
    PhaseClock clk(s, phase_seconds);
    const bool cplx = dt == CHEBFD_C128;
    CHEBFD_REQUIRE(cplx == M.complex_values, CHEBFD_EINVAL, "dtype does not match the matrix");
    const size_t es = cplx ? 16 : 8;
    const int64_t n = M.n;
    double* Y = (double*)Yv;
    Handles& h = handles_for_current_device(s);
    Buf S((size_t)ns * ns * es, s), d((size_t)ns * sizeof(double), s),
        th((size_t)ns * sizeof(double), s), Mt((size_t)ns * ns * es, s),
        T((size_t)n * ld * es, s);
    std::vector<double> hth(ns);
    int64_t counter = refill_counter ? *refill_counter : 0;
    // tall products: cuBLAS FP64, or (df) the bf16 tensor cores with the
    // FP64-accurate split of oz_gram.cu
    auto tall_gram = [&](const double* A, const double* B, double* C) {
        if (df)
            oz_gram(cplx, A, ld, B, ld, n, ns, C, M.num_sms, s);
        else
            gemm_nh(h, cplx, ns, n, A, ld, B, ld, C, ns);
    };
    auto tall_gemm = [&](int r, const double* Mc, const double* Yb, double* Tb) {
        if (df)
            oz_gemm(cplx, r, n, ns, Mc, ns, Yb, ld, Tb, ld, M.num_sms, s, true);
        else
            gemm_ch(h, cplx, r, n, ns, Mc, ns, Yb, ld, Tb, ld);
    };

    // SVQB pass on the block B (already Gram'ed into S): scale, eigensolve,
    // transform columns; returns the rank kept.
    auto svqb_transform = [&]() -> int {
        if (cplx)
            diag_scale_kernel<true><<<1, 1024, 0, s>>>(S.as<double>(), ns, d.as<double>());
        else
            diag_scale_kernel<false><<<1, 1024, 0, s>>>(S.as<double>(), ns, d.as<double>());
        heev(h, cplx, S.as<double>(), ns, th.as<double>(), s);
        CHEBFD_CHECK_CUDA(cudaMemcpyAsync(hth.data(), th.p, ns * sizeof(double),
                                          cudaMemcpyDeviceToHost, s));
        CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
        const double thr = ns * std::ldexp(1.0, -52) * hth[ns - 1];
        int first = 0;
        while (first < ns && !(hth[first] >= thr)) ++first;
        const int r = ns - first;
        CHEBFD_REQUIRE(r >= 1, CHEBFD_ENUMERIC, "orthonormalisation: block has rank 0");
        if (cplx)
            form_transform_kernel<true><<<grid1d((int64_t)ns * r), 256, 0, s>>>(
                S.as<double>(), d.as<double>(), th.as<double>(), ns, first, r, Mt.as<double>());
        else
            form_transform_kernel<false><<<grid1d((int64_t)ns * r), 256, 0, s>>>(
                S.as<double>(), d.as<double>(), th.as<double>(), ns, first, r, Mt.as<double>());
        clk.mark(PH_EIG);
        return r;
    };

    // ---- pass 1: Y1 = Y T1 (+ refill) into T
    tall_gram(Y, Y, S.as<double>());
    clk.mark(PH_GRAM);
    const int r1 = svqb_transform();
    tall_gemm(r1, Mt.as<double>(), Y, T.as<double>());
    if (r1 < ns) {
        if (cplx)
            refill_kernel<true><<<grid1d(n * (ns - r1)), 256, 0, s>>>(T.as<double>(), n, ld, r1,
                                                                      ns, counter, seed);
        else
            refill_kernel<false><<<grid1d(n * (ns - r1)), 256, 0, s>>>(T.as<double>(), n, ld, r1,
                                                                       ns, counter, seed);
        counter += ns - r1;
    }
    clk.mark(PH_BLOCK_GEMM);
    // ---- pass 2: T2 from Y1^H Y1, kept in Mt (stored conj(T2))
    tall_gram(T.as<double>(), T.as<double>(), S.as<double>());
    clk.mark(PH_GRAM);
    const int r2 = svqb_transform();
    if (r2 < ns) {
        // rank drop after pass 1: the separate, up to three-pass path
        copy_block(Y, ld, T.p, ld, n, ns, es, s);
        T.reset();
        if (refill_counter) *refill_counter = counter;
        orthonormalize_impl(Y, n, ns, ld, dt, seed, refill_counter, nullptr, s);
        if (harmonic)
            harmonic_extract(M, Y, ld, ns, cplx, tau, h, tall_gram, tall_gemm, theta_host,
                             res_host, s);
        else
            rayleigh_ritz_impl(M, Y, ld, ns, dt, theta_host, res_host, nullptr, s);
        clk.mark(PH_OTHER);
        clk.collect();
        return;
    }
    if (harmonic) {
        // Y <- Y2 = Y1 conj(Mt)
        tall_gemm(ns, Mt.as<double>(), T.as<double>(), Y);
        clk.mark(PH_BLOCK_GEMM);
        T.reset();
        harmonic_extract(M, Y, ld, ns, cplx, tau, h, tall_gram, tall_gemm, theta_host, res_host,
                         s, &clk);
        if (df) check_oz_errors(s);
        clk.collect();
        if (refill_counter) *refill_counter = counter;
        return;
    }
    // ---- Rayleigh-Ritz in the basis Y2 = Y1 T2
    Buf HY((size_t)n * ld * es, s), G((size_t)ns * ns * es, s), W2((size_t)ns * ns * es, s),
        res((size_t)ns * sizeof(double), s);
    spmv_impl(M, 1.0, 0.0, T.p, HY.p, ld, ns, dt, s);
    clk.mark(PH_HY);
    tall_gram(HY.as<double>(), T.as<double>(), G.as<double>());
    clk.mark(PH_GRAM);
    // stored conj(A2) = Mt^H conj(A1) Mt with conj(A1) in G
    gemm_small(h, cplx, false, ns, G.as<double>(), Mt.as<double>(), W2.as<double>());
    gemm_small(h, cplx, true, ns, Mt.as<double>(), W2.as<double>(), G.as<double>());
    if (cplx)
        hermitize_kernel<true><<<grid1d((int64_t)ns * ns), 256, 0, s>>>(G.as<double>(), ns);
    else
        hermitize_kernel<false><<<grid1d((int64_t)ns * ns), 256, 0, s>>>(G.as<double>(), ns);
    heev(h, cplx, G.as<double>(), ns, th.as<double>(), s);
    // C = Mt E (stored conj of T2 S); V = Y1 conj(C), HV = HY1 conj(C)
    gemm_small(h, cplx, false, ns, Mt.as<double>(), G.as<double>(), W2.as<double>());
    clk.mark(PH_EIG);
    tall_gemm(ns, W2.as<double>(), T.as<double>(), Y);
    tall_gemm(ns, W2.as<double>(), HY.as<double>(), T.as<double>());
    clk.mark(PH_BLOCK_GEMM);
    residuals_from_blocks(cplx, T.as<double>(), Y, th.as<double>(), n, ld, ns, res.as<double>(), s);
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(theta_host, th.p, ns * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
    if (res_host)
        CHEBFD_CHECK_CUDA(cudaMemcpyAsync(res_host, res.p, ns * sizeof(double),
                                          cudaMemcpyDeviceToHost, s));
    clk.mark(PH_RESIDUAL);
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
    CHEBFD_CHECK_CUDA(cudaGetLastError());
    if (df) check_oz_errors(s);
    clk.collect();
    if (refill_counter) *refill_counter = counter;
}

void residuals_impl(const Matrix& M, const void* V, const double* theta_host, int64_t ld, int k,
                    chebfd_dtype dt, double* res_host, cudaStream_t s) {
    check_fp64_block(dt, V, M.n, k, ld);
    CHEBFD_REQUIRE(theta_host && res_host, CHEBFD_EINVAL, "null argument");
    const bool cplx = dt == CHEBFD_C128;
    CHEBFD_REQUIRE(cplx == M.complex_values, CHEBFD_EINVAL, "dtype does not match the matrix");
    const size_t es = cplx ? 16 : 8;
    Buf HV((size_t)M.n * ld * es, s), th((size_t)k * sizeof(double), s),
        res((size_t)k * sizeof(double), s);
    CHEBFD_CHECK_CUDA(
        cudaMemcpyAsync(th.p, theta_host, k * sizeof(double), cudaMemcpyHostToDevice, s));
    spmv_impl(M, 1.0, 0.0, V, HV.p, ld, k, dt, s);
    residuals_from_blocks(cplx, HV.as<double>(), (const double*)V, th.as<double>(), M.n, ld, k,
                          res.as<double>(), s);
    CHEBFD_CHECK_CUDA(
        cudaMemcpyAsync(res_host, res.p, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
}

void convert_block_impl(const void* X, chebfd_dtype xdt, int64_t ldx, void* Y, chebfd_dtype ydt,
                        int64_t ldy, int64_t n, int nb, cudaStream_t s) {
    CHEBFD_REQUIRE(X && Y && n >= 1 && nb >= 1 && ldx >= nb && ldy >= nb, CHEBFD_EINVAL,
                   "bad conversion arguments");
    CHEBFD_REQUIRE(is_complex(xdt) == is_complex(ydt), CHEBFD_EINVAL,
                   "conversion keeps real/complex");
    const int rpe = is_complex(xdt) ? 2 : 1;
    const int w = nb * rpe;
    const int g = grid1d(n * w);
    const bool xs = is_single(xdt), ys = is_single(ydt);
    if (xs && !ys)
        convert_kernel<float, double><<<g, 256, 0, s>>>((const float*)X, ldx * rpe, (double*)Y,
                                                        ldy * rpe, n, w);
    else if (!xs && ys)
        convert_kernel<double, float><<<g, 256, 0, s>>>((const double*)X, ldx * rpe, (float*)Y,
                                                        ldy * rpe, n, w);
    else if (xs)
        convert_kernel<float, float><<<g, 256, 0, s>>>((const float*)X, ldx * rpe, (float*)Y,
                                                       ldy * rpe, n, w);
    else
        convert_kernel<double, double><<<g, 256, 0, s>>>((const double*)X, ldx * rpe, (double*)Y,
                                                         ldy * rpe, n, w);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

}  // namespace chebfd

using namespace chebfd;

extern "C" chebfd_status chebfd_gram(const void* A, int64_t lda, const void* B, int64_t ldb,
                                     int64_t n, int m, chebfd_dtype dt, double* C, int method,
                                     void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(A && B && C, CHEBFD_EINVAL, "null argument");
        CHEBFD_REQUIRE(dt == CHEBFD_R64 || dt == CHEBFD_C128, CHEBFD_EINVAL,
                       "the Gram product takes FP64 blocks (R64 or C128)");
        CHEBFD_REQUIRE(n >= 1 && m >= 1 && lda >= m && ldb >= m, CHEBFD_EINVAL,
                       "need n >= 1, m >= 1, lda >= m, ldb >= m");
        CHEBFD_REQUIRE(n < (1LL << 31), CHEBFD_EINVAL, "N must be < 2^31");
        const bool cplx = dt == CHEBFD_C128;
        cudaStream_t s = as_stream(stream);
        int dev = 0, sms = 0;
        CHEBFD_CHECK_CUDA(cudaGetDevice(&dev));
        CHEBFD_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        switch (method) {
            case CHEBFD_GRAM_FP64: {
                Handles& h = handles_for_current_device(s);
                gemm_nh(h, cplx, m, n, (const double*)A, lda, (const double*)B, ldb, C, m);
                break;
            }
            case CHEBFD_GRAM_DOUBLE_FLOAT: {
                Buf work(df_gram_work_bytes(m, sms), s);
                df_gram(cplx, (const double*)A, lda, (const double*)B, ldb, n, m, C, work.p, sms,
                        s);
                break;
            }
            case CHEBFD_GRAM_TENSOR:
                oz_gram(cplx, (const double*)A, lda, (const double*)B, ldb, n, m, C, sms, s);
                break;
            default:
                CHEBFD_REQUIRE(false, CHEBFD_EINVAL, "unknown Gram method");
        }
        CHEBFD_CHECK_CUDA(cudaGetLastError());
        check_oz_errors(s);
    });
}

extern "C" chebfd_status chebfd_block_update(const void* Y, int64_t ldy, int64_t n, int k,
                                             const double* M, int ldm, int r, void* T,
                                             int64_t ldt, chebfd_dtype dt, int method,
                                             void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(Y && M && T && Y != T, CHEBFD_EINVAL, "null or overlapping argument");
        CHEBFD_REQUIRE(dt == CHEBFD_R64 || dt == CHEBFD_C128, CHEBFD_EINVAL,
                       "the block update takes FP64 blocks (R64 or C128)");
        CHEBFD_REQUIRE(n >= 1 && k >= 1 && r >= 1 && ldy >= k && ldt >= r && ldm >= k,
                       CHEBFD_EINVAL, "need n, k, r >= 1, ldy >= k, ldt >= r, ldm >= k");
        CHEBFD_REQUIRE(n < (1LL << 31), CHEBFD_EINVAL, "N must be < 2^31");
        const bool cplx = dt == CHEBFD_C128;
        cudaStream_t s = as_stream(stream);
        int dev = 0, sms = 0;
        CHEBFD_CHECK_CUDA(cudaGetDevice(&dev));
        CHEBFD_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        switch (method) {
            case CHEBFD_GRAM_FP64: {
                Handles& h = handles_for_current_device(s);
                gemm_ch(h, cplx, r, n, k, M, ldm, (const double*)Y, ldy, (double*)T, ldt);
                break;
            }
            case CHEBFD_GRAM_DOUBLE_FLOAT:
                df_gemm(cplx, r, n, k, M, ldm, (const double*)Y, ldy, (double*)T, ldt, s);
                break;
            case CHEBFD_GRAM_TENSOR:
                oz_gemm(cplx, r, n, k, M, ldm, (const double*)Y, ldy, (double*)T, ldt, sms, s,
                        true);
                break;
            default:
                CHEBFD_REQUIRE(false, CHEBFD_EINVAL, "unknown method");
        }
        CHEBFD_CHECK_CUDA(cudaGetLastError());
        check_oz_errors(s);
    });
}

