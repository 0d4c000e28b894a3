// chebfd_filter_block_noalloc: the filter of chebfd_filter_block with its
// work vectors and reduction buffers in a fixed, file-scope device array
// instead of memory taken from the allocator.
//
// Some callers of this library cannot allocate device memory at the point
// where they filter: code running while another framework owns the device's
// memory through its own pool (a raw allocation there can fail or split that
// pool), and code on a latency-critical loop that must not pay for an
// allocation or its implicit synchronisation.  This entry point takes no
// device memory from anyone: the scratch below is reserved once, when the
// module is loaded on a device, and stays reserved until the process exits.
//
// The array is shared by every call on a device and keeps the contents the
// last call left there; calls whose device work overlaps (two streams, two
// host threads) race on it and must be serialised by the caller.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace chebfd {

namespace {

constexpr size_t kFlagBytes = 256;                    // completion counter + status flag
constexpr size_t kPartialBytes = (size_t)4 << 20;     // per-block moment partials
constexpr size_t kWorkBytes = (size_t)64 << 20;       // the two work vectors U and W
constexpr size_t kScratchBytes = kFlagBytes + kPartialBytes + kWorkBytes;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::once_flag g_scratch_once[kMaxDevices];
void* g_scratch_ptr[kMaxDevices] = {};
cudaError_t g_scratch_err[kMaxDevices] = {};

// Device address of g_scratch for the current device (the host-side name
// g_scratch is not a device address), looked up once per device with that
// device current; the once_flag makes concurrent first calls from several
// host threads well defined (one looks up, the others wait for it).
unsigned char* scratch_for_current_device() {
    int dev = 0;
    CHEBFD_CHECK_CUDA(cudaGetDevice(&dev));
    CHEBFD_REQUIRE(dev >= 0 && dev < kMaxDevices, CHEBFD_EUNSUPPORTED, "device index too large");
    std::call_once(g_scratch_once[dev], [dev] {
        void* p = nullptr;
        g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_scratch);
        g_scratch_ptr[dev] = p;
    });
    CHEBFD_CHECK_CUDA(g_scratch_err[dev]);
    CHEBFD_REQUIRE(g_scratch_ptr[dev] != nullptr, CHEBFD_ECUDA, "no device address for the scratch");
    return (unsigned char*)g_scratch_ptr[dev];
}

// Sets *flag to 1 if a moment is NaN/Inf or an even moment exceeds 1.001 mu_0.
__global__ void moment_check_kernel(const double* mom, int rows, int nb, int64_t ld,
                                    unsigned int* flag) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)rows * nb;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(t / nb), k = (int)(t % nb);
        const double v = mom[(int64_t)n * ld + k];
        const double mu0 = mom[k];
        bool bad = !isfinite(v);
        if (n % 2 == 0 && !(fabs(v) <= 1.001 * mu0 + 1e-300)) bad = true;
        if (bad) atomicOr(flag, 1u);
    }
}

int64_t panel_ld(chebfd_dtype dt, int nb) {
    const int64_t per = (int64_t)(16 / dtype_size(dt) > 0 ? 16 / dtype_size(dt) : 1);
    return ((nb + per - 1) / per) * per;
}

}  // namespace

int max_panel_width(chebfd_dtype dt);
void validate_block(const Matrix& M, chebfd_dtype dt, const void* X, int64_t ld, int nb);

void filter_block_noalloc_impl(const Matrix& M, double alpha, double beta, const double* gc,
                               int Np, void* X, int64_t ld, int nb, chebfd_dtype dt,
                               double* moments, cudaStream_t s) {
    validate_block(M, dt, X, ld, nb);
    CHEBFD_REQUIRE(gc != nullptr && Np >= 2, CHEBFD_EINVAL, "need Np >= 2 and coefficients");
    CHEBFD_REQUIRE(std::isfinite(alpha) && std::isfinite(beta), CHEBFD_EINVAL,
                   "alpha, beta must be finite");
    const int pw = max_panel_width(dt);
    const int wmax = std::min(pw, nb);
    const int64_t ldw = panel_ld(dt, wmax);
    const size_t es = dtype_size(dt);
    const size_t work_need = 2 * (size_t)M.n * (size_t)ldw * es;
    CHEBFD_REQUIRE(work_need <= kWorkBytes, CHEBFD_EINVAL,
                   "chebfd_filter_block_noalloc: the two work vectors need " +
                       std::to_string(work_need) + " bytes (N = " + std::to_string(M.n) +
                       ", panel width " + std::to_string(wmax) + "), more than the fixed " +
                       std::to_string(kWorkBytes) + "-byte scratch; use chebfd_filter_block");
    const size_t part_need = (size_t)M.num_sms * 8 * 2 * wmax * sizeof(double);
    CHEBFD_REQUIRE(!moments || part_need <= kPartialBytes, CHEBFD_EINVAL,
                   "chebfd_filter_block_noalloc: moment partials exceed the fixed scratch");
    unsigned char* base = scratch_for_current_device();
    unsigned int* counter = (unsigned int*)base;
    unsigned int* flag = counter + 1;
    double* partials = (double*)(base + kFlagBytes);
    char* U = (char*)(base + kFlagBytes + kPartialBytes);
    char* W = U + (size_t)M.n * ldw * es;
    // the completion counter of the moment reduction must start at zero
    CHEBFD_CHECK_CUDA(cudaMemsetAsync(base, 0, kFlagBytes, s));
    for (int p0 = 0; p0 < nb; p0 += pw) {
        const int pnb = std::min(pw, nb - p0);
        CHEBFD_REQUIRE(((size_t)pnb * es) % 16 == 0, CHEBFD_EINVAL,
                       "panel width * element size must be a multiple of 16 bytes");
        // the same panel recurrence as chebfd_filter_block, on the fixed scratch
        filter_panel(M, alpha, beta, gc, Np, (char*)X + p0 * es, ld, pnb, dt,
                     moments ? moments + p0 : nullptr, nb, U, W, ldw, partials, counter, s);
    }
    if (moments) {
        moment_check_kernel<<<64, 256, 0, s>>>(moments, 2 * Np, nb, nb, flag);
        CHEBFD_CHECK_CUDA(cudaGetLastError());
        unsigned int h = 0;
        CHEBFD_CHECK_CUDA(cudaMemcpyAsync(&h, flag, sizeof(h), cudaMemcpyDeviceToHost, s));
        CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
        CHEBFD_REQUIRE(h == 0, CHEBFD_ENUMERIC,
                       "NaN moment or diverging recurrence: spectrum not inside [a,b]");
    }
}

}  // namespace chebfd

extern "C" chebfd_status chebfd_filter_block_noalloc(const chebfd_matrix* H, double alpha,
                                                     double beta, const double* gc, int Np,
                                                     void* X, int64_t ld, int nb,
                                                     chebfd_dtype vdt, double* moments,
                                                     void* stream) {
    return chebfd::guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        chebfd::filter_block_noalloc_impl(H->m, alpha, beta, gc, Np, X, ld, nb, vdt, moments,
                                          chebfd::as_stream(stream));
    });
}
