// C ABI entry points (include/chebfd.h): error state, matrix handles, the
// coefficient construction of Sec. 2.1 and the Lanczos bounds of Sec. 3.1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <cub/cub.cuh>
#include <vector>

#include "common.cuh"

namespace chebfd {

void filter_block_impl(const Matrix& M, double alpha, double beta, const double* gc, int Np,
                       void* X, int64_t ld, int nb, chebfd_dtype dt, double* moments,
                       cudaStream_t s, int panel = 0);
void filter_block_host_impl(const Matrix& M, double alpha, double beta, const double* gc, int Np,
                            void* Xh, int64_t ld, int nb, chebfd_dtype dt, cudaStream_t s);
void spmv_impl(const Matrix& M, double alpha, double beta, const void* X, void* Y, int64_t ld,
               int nb, chebfd_dtype dt, cudaStream_t s);
void kpm_impl(const Matrix& M, double alpha, double beta, int Mm, int R, uint64_t seed,
              double* mu, cudaStream_t s);
void filter_block_df_impl(const Matrix& M, double alpha, double beta, const double* gc, int Np,
                          void* X, int64_t ld, int nb, cudaStream_t s);
void chebyshev_step_impl(const Matrix& M, double alpha, double beta, double c, const void* U,
                         void* W, void* Y, int64_t ld, int nb, chebfd_dtype dt, cudaStream_t s);

namespace {
thread_local std::string g_last_error;

void free_matrix(Matrix& m) {
    cudaFree(m.chunk_ptr);
    cudaFree(m.chunk_len);
    cudaFree(m.col);
    cudaFree(m.perm);
    cudaFree(m.val64);
    cudaFree(m.val32);
    cudaFree(m.valdf);
    cudaFree(m.bell_col);
    cudaFree(m.bell_val32);
    m = Matrix{};
}

void init_device(Matrix& m) {
    CHEBFD_CHECK_CUDA(cudaGetDevice(&m.device));
    CHEBFD_CHECK_CUDA(
        cudaDeviceGetAttribute(&m.num_sms, cudaDevAttrMultiProcessorCount, m.device));
    // Keep freed stream-ordered allocations in the pool: the filter's work
    // vectors are re-taken on every call.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, m.device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
}

// ---------------------------------------------------------------- Gershgorin

template <bool CPLX>
__global__ void gershgorin_kernel(const int64_t* chunk_ptr, const int32_t* chunk_len,
                                  const int32_t* col, const double* val, const int64_t* perm,
                                  int64_t n, int C, double* lo, double* hi) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = r / C;
        const int l = (int)(r - k * C);
        const int64_t base = chunk_ptr[k] + l;
        const int64_t orig = perm[r];
        double dre = 0.0, rad = 0.0;
        for (int j = 0; j < chunk_len[k]; ++j) {
            const int64_t pos = base + (int64_t)j * C;
            double re, im;
            if (CPLX) {
                re = val[2 * pos];
                im = val[2 * pos + 1];
            } else {
                re = val[pos];
                im = 0.0;
            }
            if (col[pos] == orig)
                dre += re;
            else
                rad += sqrt(re * re + im * im);
        }
        lo[r] = dre - rad;
        hi[r] = dre + rad;
    }
}

void gershgorin(const Matrix& M, double* glo, double* ghi, cudaStream_t s) {
    double *lo = nullptr, *hi = nullptr, *out = nullptr;
    CHEBFD_CHECK_CUDA(cudaMalloc(&lo, M.n * sizeof(double)));
    CHEBFD_CHECK_CUDA(cudaMalloc(&hi, M.n * sizeof(double)));
    CHEBFD_CHECK_CUDA(cudaMalloc(&out, 2 * sizeof(double)));
    const int g = (int)std::min<int64_t>((M.n + 255) / 256, 8192);
    if (M.complex_values)
        gershgorin_kernel<true><<<g, 256, 0, s>>>(M.chunk_ptr, M.chunk_len, M.col,
                                                  (const double*)M.val64, M.perm, M.n, M.C, lo, hi);
    else
        gershgorin_kernel<false><<<g, 256, 0, s>>>(M.chunk_ptr, M.chunk_len, M.col,
                                                   (const double*)M.val64, M.perm, M.n, M.C, lo, hi);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
    size_t b1 = 0, b2 = 0;
    cub::DeviceReduce::Min(nullptr, b1, lo, out, M.n, s);
    cub::DeviceReduce::Max(nullptr, b2, hi, out + 1, M.n, s);
    void* tmp = nullptr;
    size_t tb = std::max(b1, b2);
    CHEBFD_CHECK_CUDA(cudaMalloc(&tmp, tb + 16));
    cub::DeviceReduce::Min(tmp, tb, lo, out, M.n, s);
    tb = std::max(b1, b2);
    cub::DeviceReduce::Max(tmp, tb, hi, out + 1, M.n, s);
    double h[2];
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
    cudaFree(tmp);
    cudaFree(lo);
    cudaFree(hi);
    cudaFree(out);
    *glo = h[0];
    *ghi = h[1];
}

// ---------------------------------------------------------------- Lanczos helpers

// Deterministic FP64 reductions over single vectors stored with stride `inc`
// (in elements).  Block partials are summed in block order.
template <bool CPLX>
__global__ void dot_partials_kernel(const double* x, const double* y, int64_t n, int64_t inc,
                                    double* part) {
    __shared__ double sre[256], sim[256];
    double re = 0.0, im = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (CPLX) {
            const double xr = x[2 * i * inc], xi = x[2 * i * inc + 1];
            const double yr = y[2 * i * inc], yi = y[2 * i * inc + 1];
            re += xr * yr + xi * yi;  // conj(x) * y
            im += xr * yi - xi * yr;
        } else {
            re += x[i * inc] * y[i * inc];
        }
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sre[threadIdx.x] += sre[threadIdx.x + w];
            sim[threadIdx.x] += sim[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sre[0];
        part[2 * blockIdx.x + 1] = sim[0];
    }
}

template <bool CPLX>
__global__ void axpy_kernel(double* y, const double* x, int64_t n, int64_t inc, double ar,
                            double ai) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (CPLX) {
            const double xr = x[2 * i * inc], xi = x[2 * i * inc + 1];
            y[2 * i * inc] += ar * xr - ai * xi;
            y[2 * i * inc + 1] += ar * xi + ai * xr;
        } else {
            y[i * inc] += ar * x[i * inc];
        }
    }
}

template <bool CPLX>
__global__ void scale_copy_kernel(double* y, const double* x, int64_t n, int64_t inc, double a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (CPLX) {
            y[2 * i * inc] = a * x[2 * i * inc];
            y[2 * i * inc + 1] = a * x[2 * i * inc + 1];
        } else {
            y[i * inc] = a * x[i * inc];
        }
    }
}

template <bool CPLX>
__global__ void lanczos_start_kernel(double* v, int64_t n, int64_t inc, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (CPLX) {
            v[2 * i * inc] = 2.0 * splitmix_uniform(seed, STREAM_LANCZOS, 2 * i) - 1.0;
            v[2 * i * inc + 1] = 2.0 * splitmix_uniform(seed, STREAM_LANCZOS, 2 * i + 1) - 1.0;
        } else {
            v[i * inc] = 2.0 * splitmix_uniform(seed, STREAM_LANCZOS, i) - 1.0;
            v[i * inc + 1] = 0.0;
        }
    }
}

struct VecOps {
    int64_t n, inc;
    bool cplx;
    cudaStream_t s;
    double* part;
    std::vector<double> hpart;
    static constexpr int G = 256;
    VecOps(int64_t n_, int64_t inc_, bool c, cudaStream_t st) : n(n_), inc(inc_), cplx(c), s(st) {
        CHEBFD_CHECK_CUDA(cudaMalloc(&part, 2 * G * sizeof(double)));
        hpart.resize(2 * G);
    }
    ~VecOps() { cudaFree(part); }
    void dot(const double* x, const double* y, double* re, double* im) {
        if (cplx)
            dot_partials_kernel<true><<<G, 256, 0, s>>>(x, y, n, inc, part);
        else
            dot_partials_kernel<false><<<G, 256, 0, s>>>(x, y, n, inc, part);
        CHEBFD_CHECK_CUDA(cudaMemcpyAsync(hpart.data(), part, 2 * G * sizeof(double),
                                          cudaMemcpyDeviceToHost, s));
        CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
        double a = 0.0, b = 0.0;
        for (int i = 0; i < G; ++i) {
            a += hpart[2 * i];
            b += hpart[2 * i + 1];
        }
        *re = a;
        *im = b;
    }
    void axpy(double* y, const double* x, double ar, double ai) {
        if (cplx)
            axpy_kernel<true><<<G, 256, 0, s>>>(y, x, n, inc, ar, ai);
        else
            axpy_kernel<false><<<G, 256, 0, s>>>(y, x, n, inc, ar, ai);
        CHEBFD_CHECK_CUDA(cudaGetLastError());
    }
    void scale_copy(double* y, const double* x, double a) {
        if (cplx)
            scale_copy_kernel<true><<<G, 256, 0, s>>>(y, x, n, inc, a);
        else
            scale_copy_kernel<false><<<G, 256, 0, s>>>(y, x, n, inc, a);
        CHEBFD_CHECK_CUDA(cudaGetLastError());
    }
};

// Cyclic Jacobi eigen-decomposition of a small dense symmetric matrix
// (row-major m x m); eigenvalues ascending in w, eigenvectors in columns of Z.
void jacobi_eig(std::vector<double> A, int m, std::vector<double>& w, std::vector<double>& Z) {
    Z.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) Z[(size_t)i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                const double v = A[(size_t)i * m + j] * A[(size_t)i * m + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = A[(size_t)p * m + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) /
                                 (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; ++k) {
                    const double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
                    A[(size_t)k * m + p] = c * akp - s * akq;
                    A[(size_t)k * m + q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {
                    const double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
                    A[(size_t)p * m + k] = c * apk - s * aqk;
                    A[(size_t)q * m + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {
                    const double zkp = Z[(size_t)k * m + p], zkq = Z[(size_t)k * m + q];
                    Z[(size_t)k * m + p] = c * zkp - s * zkq;
                    Z[(size_t)k * m + q] = s * zkp + c * zkq;
                }
            }
    }
    std::vector<int> idx(m);
    for (int i = 0; i < m; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(),
              [&](int a, int b) { return A[(size_t)a * m + a] < A[(size_t)b * m + b]; });
    w.resize(m);
    std::vector<double> Zs((size_t)m * m);
    for (int j = 0; j < m; ++j) {
        w[j] = A[(size_t)idx[j] * m + idx[j]];
        for (int k = 0; k < m; ++k) Zs[(size_t)k * m + j] = Z[(size_t)k * m + idx[j]];
    }
    Z.swap(Zs);
}

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

void scale_bounds_impl(const Matrix& M, int steps, uint64_t seed, double* a_out, double* b_out,
                       cudaStream_t s) {
    CHEBFD_REQUIRE(steps >= 2, CHEBFD_EINVAL, "need at least 2 Lanczos steps");
    const bool cplx = M.complex_values;
    const chebfd_dtype dt = cplx ? CHEBFD_C128 : CHEBFD_R64;
    const int64_t ldv = cplx ? 1 : 2;  // one vector, rows padded to 16 bytes
    const int64_t n = M.n;
    const int m = (int)std::min<int64_t>(steps, n);
    const size_t vbytes = (size_t)n * ldv * 16 / (cplx ? 1 : 2);
    std::vector<double*> V(m + 1, nullptr);
    double* w = nullptr;
    auto cleanup = [&]() {
        for (auto p : V) cudaFree(p);
        cudaFree(w);
    };
    try {
        for (int j = 0; j <= m; ++j) {
            CHEBFD_CHECK_CUDA(cudaMalloc(&V[j], vbytes));
            CHEBFD_CHECK_CUDA(cudaMemsetAsync(V[j], 0, vbytes, s));
        }
        CHEBFD_CHECK_CUDA(cudaMalloc(&w, vbytes));
        CHEBFD_CHECK_CUDA(cudaMemsetAsync(w, 0, vbytes, s));
        const int64_t inc = cplx ? 1 : 2;
        VecOps ops(n, inc, cplx, s);
        if (cplx)
            lanczos_start_kernel<true><<<256, 256, 0, s>>>(V[0], n, inc, seed);
        else
            lanczos_start_kernel<false><<<256, 256, 0, s>>>(V[0], n, inc, seed);
        double re, im;
        ops.dot(V[0], V[0], &re, &im);
        ops.scale_copy(V[0], V[0], 1.0 / std::sqrt(re));
        std::vector<double> al, be;
        int k = 0;
        for (int j = 0; j < m; ++j) {
            spmv_impl(M, 1.0, 0.0, V[j], w, ldv, (int)ldv, dt, s);
            ops.dot(V[j], w, &re, &im);
            const double aj = re;
            ops.axpy(w, V[j], -aj, 0.0);
            if (j > 0) ops.axpy(w, V[j - 1], -be[j - 1], 0.0);
            for (int pass = 0; pass < 2; ++pass)  // full reorthogonalisation, twice
                for (int i = 0; i <= j; ++i) {
                    ops.dot(V[i], w, &re, &im);
                    ops.axpy(w, V[i], -re, -im);
                }
            ops.dot(w, w, &re, &im);
            const double bj = std::sqrt(std::max(re, 0.0));
            al.push_back(aj);
            be.push_back(bj);
            k = j + 1;
            if (bj == 0.0 || j == m - 1) break;
            ops.scale_copy(V[j + 1], w, 1.0 / bj);
        }
        std::vector<double> T((size_t)k * k, 0.0), th, Z;
        for (int i = 0; i < k; ++i) {
            T[(size_t)i * k + i] = al[i];
            if (i + 1 < k) T[(size_t)i * k + i + 1] = T[(size_t)(i + 1) * k + i] = be[i];
        }
        jacobi_eig(T, k, th, Z);
        const double rho_lo = std::fabs(be[k - 1] * Z[(size_t)(k - 1) * k + 0]);
        const double rho_hi = std::fabs(be[k - 1] * Z[(size_t)(k - 1) * k + (k - 1)]);
        double a = th[0] - rho_lo, b = th[k - 1] + rho_hi;
        const double width = b - a;
        a -= 0.01 * width;
        b += 0.01 * width;
        double glo, ghi;
        gershgorin(M, &glo, &ghi, s);
        *a_out = std::max(a, glo);
        *b_out = std::min(b, ghi);
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

}  // namespace chebfd

using namespace chebfd;

extern "C" {

int chebfd_abi_version(void) { return CHEBFD_ABI_VERSION; }

const char* chebfd_last_error(void) { return g_last_error.c_str(); }

const char* chebfd_status_string(chebfd_status s) {
    switch (s) {
        case CHEBFD_OK: return "ok";
        case CHEBFD_EINVAL: return "invalid argument";
        case CHEBFD_ENOMEM: return "out of memory";
        case CHEBFD_ECUDA: return "CUDA error";
        case CHEBFD_ENUMERIC: return "numerical failure";
        case CHEBFD_ENOCONV: return "not converged";
        case CHEBFD_ETIMEOUT: return "device wait timed out";
        case CHEBFD_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

chebfd_status chebfd_matrix_create_csr(int64_t n, const int64_t* rowptr, const int32_t* col,
                                       const void* val, chebfd_dtype val_dtype, int sell_C,
                                       int sell_sigma, int also_single, void* stream,
                                       chebfd_matrix** out) {
    return guarded([&] {
        CHEBFD_REQUIRE(out && rowptr && col && val, CHEBFD_EINVAL, "null argument");
        CHEBFD_REQUIRE(n >= 1 && n < (1LL << 31), CHEBFD_EINVAL, "need 1 <= n < 2^31");
        CHEBFD_REQUIRE(val_dtype == CHEBFD_R64 || val_dtype == CHEBFD_C128, CHEBFD_EINVAL,
                       "CSR values must be R64 or C128");
        CHEBFD_REQUIRE(rowptr[0] == 0, CHEBFD_EINVAL, "rowptr[0] must be 0");
        const int64_t nnz = rowptr[n];
        for (int64_t i = 0; i < n; ++i)
            CHEBFD_REQUIRE(rowptr[i + 1] >= rowptr[i], CHEBFD_EINVAL, "rowptr not monotone");
        for (int64_t k = 0; k < nnz; ++k)
            CHEBFD_REQUIRE(col[k] >= 0 && col[k] < n, CHEBFD_EINVAL, "column index out of range");
        cudaStream_t s = as_stream(stream);
        auto* h = new chebfd_matrix();
        Matrix& M = h->m;
        int64_t* d_rowptr = nullptr;
        int32_t* d_col = nullptr;
        void* d_val = nullptr;
        try {
            init_device(M);
            M.n = n;
            M.complex_values = val_dtype == CHEBFD_C128;
            const size_t vs = dtype_size(val_dtype);
            CHEBFD_CHECK_CUDA(cudaMalloc(&d_rowptr, (n + 1) * sizeof(int64_t)));
            CHEBFD_CHECK_CUDA(cudaMalloc(&d_col, std::max<int64_t>(nnz, 1) * sizeof(int32_t)));
            CHEBFD_CHECK_CUDA(cudaMalloc(&d_val, std::max<int64_t>(nnz, 1) * vs));
            CHEBFD_CHECK_CUDA(cudaMemcpyAsync(d_rowptr, rowptr, (n + 1) * sizeof(int64_t),
                                              cudaMemcpyHostToDevice, s));
            CHEBFD_CHECK_CUDA(cudaMemcpyAsync(d_col, col, nnz * sizeof(int32_t),
                                              cudaMemcpyHostToDevice, s));
            CHEBFD_CHECK_CUDA(cudaMemcpyAsync(d_val, val, nnz * vs, cudaMemcpyHostToDevice, s));
            build_sell_from_device_csr(M, d_rowptr, d_col, d_val, sell_C, sell_sigma,
                                       also_single != 0, s);
        } catch (...) {
            cudaFree(d_rowptr);
            cudaFree(d_col);
            cudaFree(d_val);
            free_matrix(M);
            delete h;
            throw;
        }
        cudaFree(d_rowptr);
        cudaFree(d_col);
        cudaFree(d_val);
        *out = h;
    });
}

chebfd_status chebfd_matrix_create_lattice(const chebfd_lattice_desc* desc, void* stream,
                                           chebfd_matrix** out) {
    return guarded([&] {
        CHEBFD_REQUIRE(desc && out, CHEBFD_EINVAL, "null argument");
        cudaStream_t s = as_stream(stream);
        auto* h = new chebfd_matrix();
        Matrix& M = h->m;
        int64_t* d_rowptr = nullptr;
        int32_t* d_col = nullptr;
        void* d_val = nullptr;
        try {
            init_device(M);
            int64_t n = 0;
            generate_lattice_csr(*desc, &n, &d_rowptr, &d_col, &d_val, s);
            M.n = n;
            M.complex_values = desc->kind != CHEBFD_LATTICE_GRAPHENE;
            build_sell_from_device_csr(M, d_rowptr, d_col, d_val, desc->sell_C,
                                       desc->sell_sigma, desc->also_single != 0, s);
            M.gen = *desc;
            M.has_gen = true;
        } catch (...) {
            cudaFree(d_rowptr);
            cudaFree(d_col);
            cudaFree(d_val);
            free_matrix(M);
            delete h;
            throw;
        }
        cudaFree(d_rowptr);
        cudaFree(d_col);
        cudaFree(d_val);
        *out = h;
    });
}

chebfd_status chebfd_matrix_get_info(const chebfd_matrix* H, chebfd_matrix_info* out) {
    return guarded([&] {
        CHEBFD_REQUIRE(H && out, CHEBFD_EINVAL, "null argument");
        const Matrix& M = H->m;
        std::memset(out, 0, sizeof(*out));
        out->n = M.n;
        out->nnz = M.nnz;
        out->nnz_padded = M.nnz_padded;
        out->nchunks = M.nchunks;
        out->C = M.C;
        out->sigma = M.sigma;
        out->max_row_len = M.max_row_len;
        out->is_complex = M.complex_values ? 1 : 0;
        out->has_single = M.val32 ? 1 : 0;
        out->blocked_width = M.bell_col ? kBellLB : 0;
    });
}

chebfd_status chebfd_matrix_set_matrix_free(chebfd_matrix* H, int enable) {
    return guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        const Matrix& M = H->m;
        const bool ok = M.has_gen && M.val32 != nullptr && M.identity_perm &&
                        (M.gen.kind == CHEBFD_LATTICE_TOPI ||
                         M.gen.kind == CHEBFD_LATTICE_TOPI_SLAB);
        CHEBFD_REQUIRE(!enable || ok, CHEBFD_EUNSUPPORTED,
                       "matrix-free step needs an insulator lattice built with also_single and "
                       "sell_sigma = 1");
        CHEBFD_REQUIRE(enable >= 0 && enable <= 2, CHEBFD_EINVAL, "mode must be 0, 1 or 2");
        H->m.stencil_enabled = enable != 0;
        H->m.stencil_pairs = enable == 2;
    });
}

chebfd_status chebfd_matrix_set_blocked(chebfd_matrix* H, int enable) {
    return guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        CHEBFD_REQUIRE(!enable || H->m.bell_col, CHEBFD_EUNSUPPORTED,
                       "matrix has no blocked copy");
        H->m.bell_enabled = enable != 0;
    });
}

chebfd_status chebfd_matrix_export_sell(const chebfd_matrix* H, int64_t* chunk_ptr,
                                        int32_t* chunk_len, int32_t* col, void* val,
                                        int64_t* perm) {
    return guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        const Matrix& M = H->m;
        if (chunk_ptr)
            CHEBFD_CHECK_CUDA(cudaMemcpy(chunk_ptr, M.chunk_ptr, (M.nchunks + 1) * sizeof(int64_t),
                                         cudaMemcpyDeviceToHost));
        if (chunk_len)
            CHEBFD_CHECK_CUDA(cudaMemcpy(chunk_len, M.chunk_len, M.nchunks * sizeof(int32_t),
                                         cudaMemcpyDeviceToHost));
        if (col)
            CHEBFD_CHECK_CUDA(
                cudaMemcpy(col, M.col, M.nnz_padded * sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (val)
            CHEBFD_CHECK_CUDA(cudaMemcpy(val, M.val64,
                                         M.nnz_padded * (M.complex_values ? 16 : 8),
                                         cudaMemcpyDeviceToHost));
        if (perm)
            CHEBFD_CHECK_CUDA(
                cudaMemcpy(perm, M.perm, M.n * sizeof(int64_t), cudaMemcpyDeviceToHost));
    });
}

chebfd_status chebfd_matrix_destroy(chebfd_matrix* H) {
    return guarded([&] {
        if (!H) return;
        free_matrix(H->m);
        delete H;
    });
}

chebfd_status chebfd_spmv(const chebfd_matrix* H, double alpha, double beta, const void* X,
                          void* Y, int64_t ld, int nb, chebfd_dtype vdt, void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        spmv_impl(H->m, alpha, beta, X, Y, ld, nb, vdt, as_stream(stream));
    });
}

chebfd_status chebfd_scale_bounds(const chebfd_matrix* H, int lanczos_steps, uint64_t seed,
                                  double* a, double* b, double* alpha, double* beta,
                                  void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        double lo, hi;
        scale_bounds_impl(H->m, lanczos_steps, seed, &lo, &hi, as_stream(stream));
        CHEBFD_REQUIRE(hi > lo, CHEBFD_ENUMERIC, "degenerate spectral interval");
        if (a) *a = lo;
        if (b) *b = hi;
        if (alpha) *alpha = 2.0 / (hi - lo);
        if (beta) *beta = (lo + hi) / (lo - hi);
    });
}

chebfd_status chebfd_window_coeffs(double a, double b, double lam_lo, double lam_hi, int Np,
                                   chebfd_kernel kernel, double mu, double* gc) {
    return guarded([&] {
        CHEBFD_REQUIRE(gc, CHEBFD_EINVAL, "null output");
        CHEBFD_REQUIRE(b > a, CHEBFD_EINVAL, "need b > a");
        CHEBFD_REQUIRE(lam_hi >= lam_lo, CHEBFD_EINVAL, "need lam_hi >= lam_lo");
        CHEBFD_REQUIRE(Np >= 1, CHEBFD_EINVAL, "need Np >= 1");
        const double pi = 3.14159265358979323846;
        const double alpha = 2.0 / (b - a), beta = (a + b) / (a - b);
        auto clamp1 = [](double x) { return x < -1.0 ? -1.0 : (x > 1.0 ? 1.0 : x); };
        const double tlo = std::acos(clamp1(alpha * lam_lo + beta));
        const double thi = std::acos(clamp1(alpha * lam_hi + beta));
        for (int n = 0; n <= Np; ++n) {
            const double c = n == 0 ? (tlo - thi) / pi
                                    : 2.0 / (pi * n) * (std::sin(n * tlo) - std::sin(n * thi));
            double g = 1.0;
            switch (kernel) {
                case CHEBFD_KERNEL_NONE: g = 1.0; break;
                case CHEBFD_KERNEL_FEJER: g = (Np - n + 1.0) / (Np + 1.0); break;
                case CHEBFD_KERNEL_JACKSON: {
                    const double q = pi / Np;
                    g = ((Np - n) * std::cos(q * n) + std::sin(q * n) / std::tan(q)) / Np;
                    break;
                }
                case CHEBFD_KERNEL_LANCZOS: {
                    if (n == 0) {
                        g = 1.0;
                    } else {
                        const double x = pi * n / (Np + 1.0);
                        g = std::pow(std::sin(x) / x, mu);
                    }
                    break;
                }
                default: throw Error{CHEBFD_EINVAL, "unknown damping kernel"};
            }
            gc[n] = g * c;
        }
    });
}

chebfd_status chebfd_filter_block(const chebfd_matrix* H, double alpha, double beta,
                                  const double* gc, int Np, void* X, int64_t ld, int nb,
                                  chebfd_dtype vdt, double* moments, void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        filter_block_impl(H->m, alpha, beta, gc, Np, X, ld, nb, vdt, moments,
                          as_stream(stream));
    });
}

chebfd_status chebfd_filter_block_host(const chebfd_matrix* H, double alpha, double beta,
                                       const double* gc, int Np, void* X_host, int64_t ld,
                                       int nb, chebfd_dtype vdt, void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        filter_block_host_impl(H->m, alpha, beta, gc, Np, X_host, ld, nb, vdt,
                               as_stream(stream));
    });
}

chebfd_status chebfd_filter_block_df(const chebfd_matrix* H, double alpha, double beta,
                                     const double* gc, int Np, void* X, int64_t ld, int nb,
                                     chebfd_dtype vdt, void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        CHEBFD_REQUIRE(vdt == (H->m.complex_values ? CHEBFD_C128 : CHEBFD_R64), CHEBFD_EINVAL,
                       "double-float filter takes the matrix's FP64 vector type");
        filter_block_df_impl(H->m, alpha, beta, gc, Np, X, ld, nb, as_stream(stream));
    });
}

chebfd_status chebfd_chebyshev_step(const chebfd_matrix* H, double alpha, double beta, double c,
                                    const void* U, void* W, void* Y, int64_t ld, int nb,
                                    chebfd_dtype vdt, void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        chebyshev_step_impl(H->m, alpha, beta, c, U, W, Y, ld, nb, vdt, as_stream(stream));
    });
}

chebfd_status chebfd_kpm_moments(const chebfd_matrix* H, double alpha, double beta, int M,
                                 int R, uint64_t seed, double* mu, void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        kpm_impl(H->m, alpha, beta, M, R, seed, mu, as_stream(stream));
    });
}

chebfd_status chebfd_random_block(void* X, int64_t n, int64_t ld, int nb, int col0,
                                  int ns_total, uint64_t seed, chebfd_dtype vdt, void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(X && n >= 1 && nb >= 1 && ld >= nb && col0 >= 0 && col0 + nb <= ns_total,
                       CHEBFD_EINVAL, "bad random block arguments");
        launch_random_block(X, n, ld, nb, col0, ns_total, seed, vdt, as_stream(stream));
    });
}

}  // extern "C"
