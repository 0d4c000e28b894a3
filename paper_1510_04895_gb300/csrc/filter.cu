// Host side of the filter path: step dispatch, the filter of Fig. ChebFD, the
// plain product Y = (alpha H + beta) X, KPM moments and random blocks.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "filter_kernels.cuh"

namespace chebfd {

void launch_step_f64(const SellView& H, bool cplx, StepMode mode, const StepArgs& a, int wc,
                     int width, int sms, cudaStream_t s);
void launch_step_f32(const SellView& H, bool cplx, StepMode mode, const StepArgs& a, int wc,
                     int width, int sms, cudaStream_t s);
bool bell_step_applies(const Matrix& M, chebfd_dtype dt, StepMode mode, const StepArgs& a,
                       int wc);
bool stencil_step_applies(const Matrix& M, chebfd_dtype dt, StepMode mode, const StepArgs& a,
                          int wc);
void launch_stencil_step(const Matrix& M, const StepArgs& a, int wc, cudaStream_t s);
void launch_bell_step(const Matrix& M, const StepArgs& a, int wc, cudaStream_t s);

namespace {

SellView view_of(const Matrix& M, bool single) {
    SellView v;
    v.chunk_ptr = M.chunk_ptr;
    v.chunk_len = M.chunk_len;
    v.col = M.col;
    v.val = single ? M.val32 : M.val64;
    v.perm = M.identity_perm ? nullptr : M.perm;
    v.n = M.n;
    v.C = M.C;
    v.logC = 0;
    while ((1 << v.logC) < M.C) ++v.logC;
    CHEBFD_REQUIRE((1 << v.logC) == M.C, CHEBFD_EINVAL, "SELL chunk height must be a power of two");
    return v;
}

// 16-byte chunks per row of an nb-wide block.
int chunks_per_row(chebfd_dtype dt, int nb) { return (int)((size_t)nb * dtype_size(dt) / 16); }

}  // namespace

int cached_occupancy(const void* kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
    int dev = 0;
    CHEBFD_CHECK_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, kernel, threads, smem);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) !=
            cudaSuccess ||
        occ < 1)
        occ = 1;
    cache[key] = occ;
    return occ;
}

void ensure_dynamic_smem(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*>, size_t> set_to;
    int dev = 0;
    CHEBFD_CHECK_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t& have = set_to[std::make_tuple(dev, kernel)];
    if (bytes <= have) return;
    CHEBFD_CHECK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)bytes));
    have = bytes;
}

SiteOrder site_order_of(const Matrix& M, int wc) {
    SiteOrder o{};
    if (!M.has_gen || M.gen.kind == CHEBFD_LATTICE_GRAPHENE || !M.identity_perm) return o;
    // In the plain order a plane's rows are gathered again (as the z-neighbours
    // of the next plane) one plane later: that needs two planes of u rows in
    // L2.  When they do not fit, visit the sites in tiles of the x-y plane,
    // all z of a tile before the next, so that z-neighbours are gathered
    // within a quarter of a wave of blocks; tile edges are the largest divisors
    // of Lx, Ly in [8, 25] (CHEBFD_SITE_TILE overrides the 25; 0 disables).
    // Measured on GB300, matrix-free step, 200x200x100 lattice: 0.79 -> 0.995
    // of HBM; 64x64x32 and 128x128x64 (whose two planes fit) stay untiled.
    static const int cap = [] {
        const char* e = getenv("CHEBFD_SITE_TILE");
        return e ? std::max(0, atoi(e)) : 25;
    }();
    static const int64_t l2 = [] {
        int dev = 0, bytes = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&bytes, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
            return (int64_t)0;
        return (int64_t)bytes;
    }();
    const int64_t window = 2LL * M.gen.Lx * M.gen.Ly * 4 * wc * 16;  // two planes of u rows
    if (cap == 0 || l2 == 0 || window <= l2) return o;
    auto tile_of = [](int L) {
        for (int t = std::min(L, cap); t >= 8; --t)
            if (L % t == 0) return t;
        return L;  // no divisor in [8, cap]: no tiling along this axis
    };
    o.Lx = M.gen.Lx;
    o.Ly = M.gen.Ly;
    o.Lz = M.gen.Lz;
    o.TX = tile_of(o.Lx);
    o.TY = tile_of(o.Ly);
    o.enabled = (o.TX < o.Lx || o.TY < o.Ly) ? 1 : 0;
    return o;
}

int max_panel_width(chebfd_dtype dt) {
    // 64 chunks of 16 bytes per row group: 64 complex doubles, 128 complex floats,
    // 128 doubles, 256 floats; kept at 64 / 128 to bound register use.
    switch (dt) {
        case CHEBFD_C128: return 32;  // FP64-ALU bound: narrower panels keep the fast path
        case CHEBFD_C64: return 64;
        case CHEBFD_R64: return 128;
        case CHEBFD_R32: return 128;
    }
    return 0;
}

void validate_block(const Matrix& M, chebfd_dtype dt, const void* X, int64_t ld, int nb) {
    CHEBFD_REQUIRE(X != nullptr, CHEBFD_EINVAL, "null block pointer");
    CHEBFD_REQUIRE(nb >= 1 && ld >= nb, CHEBFD_EINVAL, "need 1 <= nb <= ld");
    CHEBFD_REQUIRE(is_complex(dt) == M.complex_values, CHEBFD_EINVAL,
                   "vector dtype must match the matrix (complex vs real)");
    CHEBFD_REQUIRE(!is_single(dt) || M.val32 != nullptr, CHEBFD_EINVAL,
                   "single-precision vectors need a matrix built with also_single");
    CHEBFD_REQUIRE(((uintptr_t)X % 16) == 0, CHEBFD_EINVAL, "block base must be 16-byte aligned");
    CHEBFD_REQUIRE(((size_t)ld * dtype_size(dt)) % 16 == 0, CHEBFD_EINVAL,
                   "ld * element size must be a multiple of 16 bytes");
    CHEBFD_REQUIRE(((size_t)nb * dtype_size(dt)) % 16 == 0, CHEBFD_EINVAL,
                   "nb * element size must be a multiple of 16 bytes");
}

void launch_step(const Matrix& M, chebfd_dtype dt, StepMode mode, const StepArgs& a,
                 cudaStream_t stream) {
    const int wc = chunks_per_row(dt, a.nb);
    CHEBFD_REQUIRE(wc >= 1 && wc <= 64, CHEBFD_EINVAL, "panel too wide for one row group");
    if (stencil_step_applies(M, dt, mode, a, wc)) {
        StepArgs b = a;
        b.order = site_order_of(M, wc);
        launch_stencil_step(M, b, wc, stream);
        return;
    }
    if (bell_step_applies(M, dt, mode, a, wc)) {
        StepArgs b = a;
        b.order = a.coef ? SiteOrder{} : site_order_of(M, wc);
        launch_bell_step(M, b, wc, stream);
        CHEBFD_CHECK_CUDA(cudaGetLastError());
        return;
    }
    const SellView v = view_of(M, is_single(dt));
    StepArgs args = a;
    if (args.tile <= 0) {
        static const int env_tile = [] {
            const char* e = getenv("CHEBFD_STEP_TILE");
            return e ? std::max(1, atoi(e)) : 4;
        }();
        args.tile = env_tile;
    }
    // persistent grid: resident blocks per SM (occupancy) x SM count
    if (is_single(dt))
        launch_step_f32(v, is_complex(dt), mode, args, wc, M.uniform_width, M.num_sms, stream);
    else
        launch_step_f64(v, is_complex(dt), mode, args, wc, M.uniform_width, M.num_sms, stream);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------ random blocks

namespace {

template <class R, bool CPLX>
__global__ void random_block_kernel(R* X, int64_t n, int64_t ld, int nb, int col0, int ns_total,
                                    uint64_t seed) {
    const int64_t total = n * nb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / nb;
        const int k = (int)(t - i * nb);
        const uint64_t idx = (uint64_t)i * (uint64_t)ns_total + (uint64_t)(k + col0);
        if (CPLX) {
            const double re = 2.0 * splitmix_uniform(seed, STREAM_SEARCH, 2 * idx) - 1.0;
            const double im = 2.0 * splitmix_uniform(seed, STREAM_SEARCH, 2 * idx + 1) - 1.0;
            X[2 * (i * ld + k)] = (R)re;
            X[2 * (i * ld + k) + 1] = (R)im;
        } else {
            X[i * ld + k] = (R)(2.0 * splitmix_uniform(seed, STREAM_SEARCH, idx) - 1.0);
        }
    }
}

template <class R, bool CPLX>
__global__ void kpm_probe_kernel(R* X, int64_t n, int64_t ld, int R_, uint64_t seed) {
    const int64_t total = n * R_;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / R_;
        const int r = (int)(t - i * R_);
        const uint64_t w = splitmix_word(seed, STREAM_KPM, (uint64_t)t);
        const double s0 = (w & 1ULL) ? -1.0 : 1.0;
        if (CPLX) {
            const double s1 = (w & 2ULL) ? -1.0 : 1.0;
            const double h = 0.70710678118654752440;  // 1/sqrt(2), correctly rounded
            X[2 * (i * ld + r)] = (R)(s0 * h);
            X[2 * (i * ld + r) + 1] = (R)(s1 * h);
        } else {
            X[i * ld + r] = (R)s0;
        }
    }
}

int small_grid(int64_t work) {
    int64_t g = (work + 255) / 256;
    return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 4096);
}

}  // namespace

void launch_random_block(void* X, int64_t n, int64_t ld, int nb, int col0, int ns_total,
                         uint64_t seed, chebfd_dtype dt, cudaStream_t s) {
    const int g = small_grid(n * nb);
    switch (dt) {
        case CHEBFD_R64:
            random_block_kernel<double, false><<<g, 256, 0, s>>>((double*)X, n, ld, nb, col0, ns_total, seed);
            break;
        case CHEBFD_C128:
            random_block_kernel<double, true><<<g, 256, 0, s>>>((double*)X, n, ld, nb, col0, ns_total, seed);
            break;
        case CHEBFD_R32:
            random_block_kernel<float, false><<<g, 256, 0, s>>>((float*)X, n, ld, nb, col0, ns_total, seed);
            break;
        case CHEBFD_C64:
            random_block_kernel<float, true><<<g, 256, 0, s>>>((float*)X, n, ld, nb, col0, ns_total, seed);
            break;
    }
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

void launch_kpm_probes(void* X, int64_t n, int64_t ld, int R, uint64_t seed, chebfd_dtype dt,
                       cudaStream_t s) {
    const int g = small_grid(n * R);
    switch (dt) {
        case CHEBFD_R64: kpm_probe_kernel<double, false><<<g, 256, 0, s>>>((double*)X, n, ld, R, seed); break;
        case CHEBFD_C128: kpm_probe_kernel<double, true><<<g, 256, 0, s>>>((double*)X, n, ld, R, seed); break;
        case CHEBFD_R32: kpm_probe_kernel<float, false><<<g, 256, 0, s>>>((float*)X, n, ld, R, seed); break;
        case CHEBFD_C64: kpm_probe_kernel<float, true><<<g, 256, 0, s>>>((float*)X, n, ld, R, seed); break;
    }
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------ workspace

namespace {

struct DeviceBuffer {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    DeviceBuffer(size_t bytes, cudaStream_t stream) : s(stream) {
        if (bytes) CHEBFD_CHECK_CUDA(cudaMallocAsync(&p, bytes, stream));
    }
    ~DeviceBuffer() {
        if (p) cudaFreeAsync(p, s);
    }
    DeviceBuffer(const DeviceBuffer&) = delete;
    DeviceBuffer& operator=(const DeviceBuffer&) = delete;
};

int64_t padded_ld(chebfd_dtype dt, int nb) {
    const size_t per = 16 / std::min<size_t>(16, dtype_size(dt));
    return ((nb + (int64_t)per - 1) / (int64_t)per) * (int64_t)per;
}

}  // namespace

// One panel of the filter p[H] X = sum_n g_n c_n T_n(A) X, A = alpha H + beta
// (Sec. 2.1), evaluated by the Chebyshev three-term recurrence in the order of
// Fig. ChebFD: U and W (workspace panels, leading dimension ldw) hold the two
// most recent T_n(A) X, and the panel X itself becomes the accumulated sum.
void filter_panel(const Matrix& M, double alpha, double beta, const double* gc, int Np, char* X,
                  int64_t ld, int nb, chebfd_dtype dt, double* moments, int64_t mom_ld,
                  char* U, char* W, int64_t ldw, double* partials, unsigned int* counter,
                  cudaStream_t s, char* W2, char* W3) {
    StepArgs a{};
    a.nb = nb;
    a.alpha = alpha;
    a.beta = beta;
    a.partials = partials;
    a.counter = counter;
    a.moments = moments;
    a.mom_ld = mom_ld;
    // T_1 = A T_0 with T_0 = X, into U
    a.gather = X;
    a.ldg = ld;
    a.w = U;
    a.ldw = ldw;
    a.y = nullptr;
    a.ldy = 0;
    a.mom_step = 1;
    launch_step(M, dt, MODE_SPMV, a, s);
    // T_2 = 2 A T_1 - T_0 into W; the sum starts as gc_0 T_0 + gc_1 T_1 + gc_2 T_2 in X
    a.gather = U;
    a.ldg = ldw;
    a.w = W;
    a.ldw = ldw;
    a.y = X;
    a.ldy = ld;
    a.c0 = gc[0];
    a.c1 = gc[1];
    a.c2 = gc[2];
    a.mom_step = 2;
    launch_step(M, dt, MODE_SECOND, a, s);
    // n = 3..Np: T_n = 2 A T_{n-1} - T_{n-2} overwrites the buffer of T_{n-2};
    // the sum gains gc_n T_n in the same pass
    char* t_prev = U;  // T_{n-2}
    char* t_cur = W;   // T_{n-1}
    int n0 = 3;
    if (W2 && W3 && !moments && stencil2_applies(M, dt, nb)) {
        // pairs: T_n, T_{n+1} into the two spare panels, which then become
        // the latest two; the older two are the spares of the next pair
        char* s1 = W2;
        char* s2 = W3;
        for (; n0 + 1 <= Np; n0 += 2) {
            launch_stencil2(M, t_cur, t_prev, s1, s2, X, ldw, ld, alpha, beta, gc[n0], gc[n0 + 1],
                            s);
            std::swap(t_prev, s1);
            std::swap(t_cur, s2);
        }
    }
    for (int n = n0; n <= Np; ++n) {
        a.gather = t_cur;
        a.w = t_prev;  // T_{n-2} in, T_n out
        a.c0 = gc[n];
        a.mom_step = n;
        launch_step(M, dt, MODE_STEP, a, s);
        std::swap(t_prev, t_cur);
    }
}

void filter_block_impl(const Matrix& M, double alpha, double beta, const double* gc, int Np,
                       void* X, int64_t ld, int nb, chebfd_dtype dt, double* moments,
                       cudaStream_t s, int panel) {
    validate_block(M, dt, X, ld, nb);
    CHEBFD_REQUIRE(gc != nullptr && Np >= 2, CHEBFD_EINVAL, "need Np >= 2 and coefficients");
    CHEBFD_REQUIRE(std::isfinite(alpha) && std::isfinite(beta), CHEBFD_EINVAL,
                   "alpha, beta must be finite");
    int pw = panel > 0 ? std::min(panel, max_panel_width(dt)) : max_panel_width(dt);
    // the matrix-free insulator: 16-column panels, two steps per pass
    const bool pairs = !moments && nb >= 16 && nb % 16 == 0 && stencil2_applies(M, dt, 16);
    if (pairs) pw = 16;
    const int wmax = std::min(pw, nb);
    const int64_t ldw = padded_ld(dt, wmax);
    const size_t es = dtype_size(dt);
    DeviceBuffer U((size_t)M.n * ldw * es, s), W((size_t)M.n * ldw * es, s);
    DeviceBuffer W2(pairs ? (size_t)M.n * ldw * es : 0, s), W3(pairs ? (size_t)M.n * ldw * es : 0, s);
    const int grid_max = M.num_sms * 8;
    DeviceBuffer part(moments ? (size_t)grid_max * 2 * wmax * sizeof(double) : 0, s);
    DeviceBuffer cnt(moments ? 256 : 0, s);
    if (moments) CHEBFD_CHECK_CUDA(cudaMemsetAsync(cnt.p, 0, 256, s));
    for (int p0 = 0; p0 < nb; p0 += pw) {
        const int pnb = std::min(pw, nb - p0);
        CHEBFD_REQUIRE(((size_t)pnb * es) % 16 == 0, CHEBFD_EINVAL,
                       "panel width * element size must be a multiple of 16 bytes");
        filter_panel(M, alpha, beta, gc, Np, (char*)X + p0 * es, ld, pnb, dt,
                     moments ? moments + p0 : nullptr, nb, (char*)U.p, (char*)W.p, ldw,
                     (double*)part.p, (unsigned int*)cnt.p, s, (char*)W2.p, (char*)W3.p);
    }
    if (moments) {
        std::vector<double> h((size_t)2 * Np * nb);
        CHEBFD_CHECK_CUDA(cudaMemcpyAsync(h.data(), moments, h.size() * sizeof(double),
                                          cudaMemcpyDeviceToHost, s));
        CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < nb; ++k) {
            const double mu0 = h[k];
            for (int n = 0; n < 2 * Np; ++n) {
                const double v = h[(size_t)n * nb + k];
                CHEBFD_REQUIRE(std::isfinite(v), CHEBFD_ENUMERIC, "NaN/Inf Chebyshev moment");
                if (n % 2 == 0)
                    CHEBFD_REQUIRE(std::fabs(v) <= 1.001 * mu0 + 1e-300, CHEBFD_ENUMERIC,
                                   "Chebyshev recurrence diverged: spectrum not inside [a,b]");
            }
        }
    }
}

namespace {

// The two copy streams of a device (to and from the host), created once.
struct CopyStreams {
    cudaStream_t h2d = nullptr, d2h = nullptr;
};

CopyStreams& copy_streams() {
    static std::once_flag once[64];
    static CopyStreams cs[64];
    int dev = 0;
    CHEBFD_CHECK_CUDA(cudaGetDevice(&dev));
    CHEBFD_REQUIRE(dev >= 0 && dev < 64, CHEBFD_ECUDA, "device index out of range");
    std::call_once(once[dev], [dev] {
        CHEBFD_CHECK_CUDA(cudaStreamCreateWithFlags(&cs[dev].h2d, cudaStreamNonBlocking));
        CHEBFD_CHECK_CUDA(cudaStreamCreateWithFlags(&cs[dev].d2h, cudaStreamNonBlocking));
    });
    return cs[dev];
}

// Events owned for the length of one call (destroyed when it returns; the
// runtime releases an event still pending once it completes).
struct EventSet {
    std::vector<cudaEvent_t> e;
    void create(int n) {
        e.assign(n, nullptr);
        for (auto& x : e) CHEBFD_CHECK_CUDA(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
    }
    ~EventSet() {
        for (auto x : e)
            if (x) cudaEventDestroy(x);
    }
};

}  // namespace

// The filter of a host-resident block, streamed through the device panel by
// panel (same panels and kernels as filter_block_impl, so the same result):
// a ring of up to three device panels; panel p is copied in on the h2d
// stream, filtered on s, copied back on the d2h stream, and its buffer is
// refilled (panel p + 3) only after that copy-out has completed.
void filter_block_host_impl(const Matrix& M, double alpha, double beta, const double* gc, int Np,
                            void* Xh, int64_t ld, int nb, chebfd_dtype dt, cudaStream_t s) {
    validate_block(M, dt, Xh, ld, nb);
    CHEBFD_REQUIRE(gc != nullptr && Np >= 2, CHEBFD_EINVAL, "need Np >= 2 and coefficients");
    CHEBFD_REQUIRE(std::isfinite(alpha) && std::isfinite(beta), CHEBFD_EINVAL,
                   "alpha, beta must be finite");
    const int pw = max_panel_width(dt);
    const int np = (nb + pw - 1) / pw, nbuf = std::min(np, 3);
    const int64_t ldp = padded_ld(dt, std::min(pw, nb));
    const size_t es = dtype_size(dt), panel_bytes = (size_t)M.n * ldp * es;
    DeviceBuffer P(panel_bytes * nbuf, s), U(panel_bytes, s), W(panel_bytes, s);
    CopyStreams& cs = copy_streams();
    EventSet ev;
    ev.create(1 + 3 * np);
    auto h2d_done = [&](int p) { return ev.e[1 + 3 * p]; };
    auto filtered = [&](int p) { return ev.e[2 + 3 * p]; };
    auto d2h_done = [&](int p) { return ev.e[3 + 3 * p]; };
    // the copy streams start after the allocations and earlier work on s
    CHEBFD_CHECK_CUDA(cudaEventRecord(ev.e[0], s));
    CHEBFD_CHECK_CUDA(cudaStreamWaitEvent(cs.h2d, ev.e[0], 0));
    CHEBFD_CHECK_CUDA(cudaStreamWaitEvent(cs.d2h, ev.e[0], 0));
    for (int p = 0; p < np; ++p) {
        const int p0 = p * pw, pnb = std::min(pw, nb - p0);
        char* buf = (char*)P.p + (size_t)(p % nbuf) * panel_bytes;
        char* host = (char*)Xh + (size_t)p0 * es;
        if (p >= nbuf) CHEBFD_CHECK_CUDA(cudaStreamWaitEvent(cs.h2d, d2h_done(p - nbuf), 0));
        CHEBFD_CHECK_CUDA(cudaMemcpy2DAsync(buf, ldp * es, host, ld * es, pnb * es, M.n,
                                            cudaMemcpyHostToDevice, cs.h2d));
        CHEBFD_CHECK_CUDA(cudaEventRecord(h2d_done(p), cs.h2d));
        CHEBFD_CHECK_CUDA(cudaStreamWaitEvent(s, h2d_done(p), 0));
        filter_panel(M, alpha, beta, gc, Np, buf, ldp, pnb, dt, nullptr, 0, (char*)U.p,
                     (char*)W.p, ldp, nullptr, nullptr, s, nullptr, nullptr);
        CHEBFD_CHECK_CUDA(cudaEventRecord(filtered(p), s));
        CHEBFD_CHECK_CUDA(cudaStreamWaitEvent(cs.d2h, filtered(p), 0));
        CHEBFD_CHECK_CUDA(cudaMemcpy2DAsync(host, ld * es, buf, ldp * es, pnb * es, M.n,
                                            cudaMemcpyDeviceToHost, cs.d2h));
        CHEBFD_CHECK_CUDA(cudaEventRecord(d2h_done(p), cs.d2h));
    }
    // the caller's stream (and the panel buffers' release on it) waits for
    // the last copy-out, which follows every earlier one on the d2h stream
    CHEBFD_CHECK_CUDA(cudaStreamWaitEvent(s, d2h_done(np - 1), 0));
}

void spmv_impl(const Matrix& M, double alpha, double beta, const void* X, void* Y, int64_t ld,
               int nb, chebfd_dtype dt, cudaStream_t s) {
    validate_block(M, dt, X, ld, nb);
    validate_block(M, dt, Y, ld, nb);
    CHEBFD_REQUIRE(X != Y, CHEBFD_EINVAL, "spmv needs Y != X");
    const int pw = max_panel_width(dt);
    const size_t es = dtype_size(dt);
    for (int p0 = 0; p0 < nb; p0 += pw) {
        StepArgs a{};
        a.nb = std::min(pw, nb - p0);
        a.alpha = alpha;
        a.beta = beta;
        a.gather = (const char*)X + p0 * es;
        a.ldg = ld;
        a.w = (char*)Y + p0 * es;
        a.ldw = ld;
        launch_step(M, dt, MODE_SPMV, a, s);
    }
}

void chebyshev_step_impl(const Matrix& M, double alpha, double beta, double c, const void* U,
                         void* W, void* Y, int64_t ld, int nb, chebfd_dtype dt, cudaStream_t s) {
    validate_block(M, dt, U, ld, nb);
    validate_block(M, dt, W, ld, nb);
    validate_block(M, dt, Y, ld, nb);
    CHEBFD_REQUIRE(U != W && U != Y && W != Y, CHEBFD_EINVAL, "U, W, Y must be distinct");
    CHEBFD_REQUIRE(nb <= max_panel_width(dt), CHEBFD_EINVAL, "nb wider than one row group");
    StepArgs a{};
    a.nb = nb;
    a.alpha = alpha;
    a.beta = beta;
    a.c0 = c;
    a.gather = U;
    a.ldg = ld;
    a.w = W;
    a.ldw = ld;
    a.y = Y;
    a.ldy = ld;
    launch_step(M, dt, MODE_STEP, a, s);
}

void kpm_impl(const Matrix& M, double alpha, double beta, int Mm, int R, uint64_t seed,
              double* mu, cudaStream_t s) {
    CHEBFD_REQUIRE(Mm >= 2 && Mm % 2 == 0, CHEBFD_EINVAL, "M must be even and >= 2");
    CHEBFD_REQUIRE(R >= 1, CHEBFD_EINVAL, "need R >= 1 probe vectors");
    CHEBFD_REQUIRE(mu != nullptr, CHEBFD_EINVAL, "null output");
    const chebfd_dtype dt = M.complex_values ? CHEBFD_C128 : CHEBFD_R64;
    const int Np = Mm / 2;
    // Probes go through the filter with gc = 0 (only the moments are kept).
    const int64_t ld = padded_ld(dt, R);
    const size_t es = dtype_size(dt);
    DeviceBuffer X((size_t)M.n * ld * es, s);
    CHEBFD_CHECK_CUDA(cudaMemsetAsync(X.p, 0, (size_t)M.n * ld * es, s));
    launch_kpm_probes(X.p, M.n, ld, R, seed, dt, s);
    DeviceBuffer mom((size_t)2 * std::max(Np, 2) * ld * sizeof(double), s);
    std::vector<double> gc(std::max(Np, 2) + 1, 0.0);
    // The padded columns are zero vectors: their moments are 0 and are ignored.
    filter_block_impl(M, alpha, beta, gc.data(), std::max(Np, 2), X.p, ld, (int)ld, dt,
                      (double*)mom.p, s, 0);
    std::vector<double> h((size_t)2 * std::max(Np, 2) * ld);
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(h.data(), mom.p, h.size() * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
    for (int n = 0; n < Mm; ++n) {
        double acc = 0.0;
        for (int r = 0; r < R; ++r) acc += h[(size_t)n * ld + r];
        mu[n] = acc / ((double)R * (double)M.n);
    }
}

}  // namespace chebfd
