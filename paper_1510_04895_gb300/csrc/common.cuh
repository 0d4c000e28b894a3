// Internal declarations shared by the translation units of libchebfd.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/chebfd.h"

namespace chebfd {

// ---------------------------------------------------------------- errors

void set_error(const std::string& msg);

struct Error {
    chebfd_status code;
    std::string msg;
};

#define CHEBFD_CHECK_CUDA(expr)                                                       \
    do {                                                                              \
        cudaError_t e_ = (expr);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            throw ::chebfd::Error{e_ == cudaErrorMemoryAllocation ? CHEBFD_ENOMEM     \
                                                                   : CHEBFD_ECUDA,    \
                                  std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
        }                                                                             \
    } while (0)

#define CHEBFD_REQUIRE(cond, code, msg)                               \
    do {                                                              \
        if (!(cond)) throw ::chebfd::Error{(code), std::string(msg)}; \
    } while (0)

// Run `body` and translate exceptions into a status + thread-local message.
template <class F>
chebfd_status guarded(F&& body) {
    try {
        body();
        return CHEBFD_OK;
    } catch (const Error& e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return CHEBFD_ENOMEM;
    } catch (const std::exception& e) {
        set_error(e.what());
        return CHEBFD_ECUDA;
    }
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool is_complex(chebfd_dtype d) { return d == CHEBFD_C128 || d == CHEBFD_C64; }
inline bool is_single(chebfd_dtype d) { return d == CHEBFD_R32 || d == CHEBFD_C64; }
inline size_t dtype_size(chebfd_dtype d) {
    switch (d) {
        case CHEBFD_R64: return 8;
        case CHEBFD_C128: return 16;
        case CHEBFD_R32: return 4;
        case CHEBFD_C64: return 8;
    }
    return 0;
}

// ---------------------------------------------------------------- matrix

// Device SELL-C-sigma storage (column-major inside chunks of C rows).
struct Matrix {
    int64_t n = 0;
    int64_t nnz = 0;
    int64_t nnz_padded = 0;
    int64_t nchunks = 0;
    int C = 1, sigma = 1;
    int max_row_len = 0;
    int uniform_width = 0;  // > 0: every chunk has this width (ELLPACK shape)
    bool complex_values = false;
    bool identity_perm = true;
    int64_t* chunk_ptr = nullptr;  // [nchunks+1]
    int32_t* chunk_len = nullptr;  // [nchunks]
    int32_t* col = nullptr;        // [nnz_padded]
    int64_t* perm = nullptr;       // [n], original row of sorted row r
    void* val64 = nullptr;         // double or double2 [nnz_padded]
    void* val32 = nullptr;         // float or float2 [nnz_padded], optional
    // Double-float copy of the values [nnz_padded], built with val32: complex
    // float4 (re_hi, re_lo, im_hi, im_lo), real float2 (hi, lo).
    void* valdf = nullptr;
    // Blocked-ELL copy of a complex matrix whose rows fall into blocks of
    // kBellB consecutive rows that couple to at most kBellLB blocks of
    // columns each (the 4 orbitals of a lattice site and its 6 neighbours):
    // bell_col[nbr][kBellLB] block columns (slot 0 is the own block row,
    // unused slots repeat it with zero values), bell_val32[nbr][kBellLB][b][b]
    // dense complex64 blocks, row-major.  Built only with also_single and
    // identity row order; used by the single-precision step kernel.
    int32_t* bell_col = nullptr;
    void* bell_val32 = nullptr;
    bool bell_enabled = false;
    // Generator of a lattice matrix (has_gen), for the matrix-free insulator
    // step that rebuilds the entries in registers (stencil_enabled).
    chebfd_lattice_desc gen{};
    bool has_gen = false;
    bool stencil_enabled = false;
    bool stencil_pairs = false;   // two Chebyshev steps per pass (16-column panels)
    // Row panel order used by the kernels (same as sorted order here).
    int device = 0;
    int num_sms = 0;
};

constexpr int kBellB = 4;   // rows per block (orbitals per site)
constexpr int kBellLB = 7;  // block columns per block row (own site + 6 neighbours)

// Build the SELL arrays from a device CSR (rowptr[n+1], col, FP64 values).
// Takes ownership of nothing; the CSR buffers may be freed afterwards.
void build_sell_from_device_csr(Matrix& M, const int64_t* d_rowptr, const int32_t* d_col,
                                const void* d_val, int C, int sigma, bool also_single,
                                cudaStream_t stream);

// Resident blocks per SM of a kernel at `threads` threads and `smem` dynamic
// shared bytes on the current device (occupancy API, cached per kernel); >= 1.
int cached_occupancy(const void* kernel, int threads, size_t smem);

// The kernel may use `bytes` of dynamic shared memory on the current device
// (cudaFuncSetAttribute once per device and kernel; thread-safe).
void ensure_dynamic_smem(const void* kernel, size_t bytes);

// Keep the library's stream-ordered workspace cached between calls (oz_gram.cu).
void cache_stream_workspace();

// Blocked-ELL copy (bell_col, bell_val32) when the CSR has that shape; no-op otherwise.
void build_bell(Matrix& M, const int64_t* d_rowptr, const int32_t* d_col, const double* d_val,
                cudaStream_t stream);

void generate_lattice_csr(const chebfd_lattice_desc& d, int64_t* n_out, int64_t** d_rowptr,
                          int32_t** d_col, void** d_val, cudaStream_t stream);

// ---------------------------------------------------------------- kernels

enum StepMode { MODE_SPMV = 0, MODE_SECOND = 1, MODE_STEP = 2 };

// Visiting order of the sites of an Lx x Ly x Lz lattice (4 rows per site)
// for the step kernels: tiles of TX x TY sites of the x-y plane, all z of a
// tile before the next tile, so that the z-neighbours of a tile are gathered
// while still in L2 (a whole 200 x 200 plane of a 64-column complex64 block
// is 82 MB).  Visit index q -> site.  TX | Lx and TY | Ly; enabled == 0: q is
// the site itself.
struct SiteOrder {
    int enabled;
    int Lx, Ly, Lz, TX, TY;
    __device__ __forceinline__ int64_t site(int64_t q) const {
        if (!enabled) return q;
        const int qi = (int)q;  // < 2^29 sites
        const int plane = TX * TY, per_tile = plane * Lz;
        const int tile = qi / per_tile, rem = qi - tile * per_tile;
        const int z = rem / plane, l = rem - z * plane;
        const int ly = l / TX, lx = l - ly * TX;
        const int ntx = Lx / TX;
        const int ty = tile / ntx, tx = tile - ty * ntx;
        return (int64_t)(tx * TX + lx) + (int64_t)Lx * ((ty * TY + ly) + (int64_t)Ly * z);
    }
};

struct StepArgs {
    // Vectors (row-major, ld elements per row).
    const void* gather;  // u: gathered through H (input of the product)
    void* w;             // MODE_SPMV: output; MODE_SECOND: output w; MODE_STEP: in/out w
    void* y;             // MODE_SECOND/STEP: accumulated block (in/out); unused for SPMV
    int64_t ldg, ldw, ldy;  // leading dimensions (elements) of gather, w, y
    int nb;
    double alpha, beta;  // A = alpha H + beta
    double c0, c1, c2;   // MODE_SECOND: y = c0 x + c1 u + c2 w ; MODE_STEP: y += c0 w
    // Moments (optional): device partial buffer and output.
    double* partials;    // [grid * 2 * nb]
    unsigned int* counter;
    double* moments;     // [2*Np x mom_ld]; nullptr = no dots
    int64_t mom_ld;
    int mom_step;        // n of the step: writes mu_{2n-2}, mu_{2n-1} (SPMV: mu_0, mu_1)
    int tile;            // consecutive row groups per block and wave (0 = 1)
    // Ensemble of independent matrices (block-diagonal): per-instance
    // coefficients coef[inst * coef_ld + {0: alpha, 1: beta, 2 + n: gc_n,
    // coef_ld - 1: beta / alpha (diagonal shift of the blocked step)}],
    // instance of each (original) row in row_inst.  nullptr: single matrix.
    const double* coef;
    const int32_t* row_inst;
    int coef_ld;
    SiteOrder order;     // site visiting order of lattice matrices (set by launch_step)
};

// The site order for a generated insulator lattice and a panel of wc
// 16-byte chunks per row (tiled when two planes of u rows exceed L2).
SiteOrder site_order_of(const Matrix& M, int wc);

// Launch one step kernel.  dt selects the vector type, `single` the matrix copy.
void launch_step(const Matrix& M, chebfd_dtype dt, StepMode mode, const StepArgs& a,
                 cudaStream_t stream);
int max_panel_width(chebfd_dtype dt);

// Phases of the dense steps (Sec. 3.1 steps 6-7) timed with CUDA events on the
// solve's stream: tall Gram products, tall block products, the n_s x n_s
// eigenproblems with their small products and host decisions, the products
// H Y, the residual norms, and anything else (rank-drop fallbacks).
enum DensePhase { PH_GRAM = 0, PH_BLOCK_GEMM, PH_EIG, PH_HY, PH_RESIDUAL, PH_OTHER, PH_COUNT };

// Records an event at each phase boundary; collect() waits for the last one
// and adds each segment's time to acc[phase].  acc == nullptr: no events.
class PhaseClock {
  public:
    PhaseClock(cudaStream_t s, double* acc) : s_(s), acc_(acc) { record(-1); }
    ~PhaseClock() { release(); }
    PhaseClock(const PhaseClock&) = delete;
    PhaseClock& operator=(const PhaseClock&) = delete;
    // the work enqueued since the previous mark belongs to `phase`
    void mark(int phase) { record(phase); }
    void collect() {
        if (!acc_ || ev_.size() < 2) return;
        CHEBFD_CHECK_CUDA(cudaEventSynchronize(ev_.back()));
        for (size_t i = 1; i < ev_.size(); ++i) {
            float ms = 0.f;
            CHEBFD_CHECK_CUDA(cudaEventElapsedTime(&ms, ev_[i - 1], ev_[i]));
            acc_[ph_[i]] += 1e-3 * ms;
        }
        release();
        record(-1);
    }

  private:
    void record(int phase) {
        if (!acc_) return;
        cudaEvent_t e = nullptr;
        CHEBFD_CHECK_CUDA(cudaEventCreate(&e));
        ev_.push_back(e);
        ph_.push_back(phase);
        CHEBFD_CHECK_CUDA(cudaEventRecord(e, s_));
    }
    void release() {
        for (cudaEvent_t e : ev_) cudaEventDestroy(e);
        ev_.clear();
        ph_.clear();
    }
    cudaStream_t s_;
    double* acc_;
    std::vector<cudaEvent_t> ev_;
    std::vector<int> ph_;
};

// One panel (nb <= max_panel_width) of p[H] X by the Chebyshev recurrence:
// X (ld) becomes sum_n gc[n] T_n(A) X; U, W are two work panels (ldw);
// moments (nullable, 2 Np x mom_ld) with per-block partials and a completion
// counter that starts at zero.  Asynchronous on s.
// With two more work panels W2, W3 (non-null) and a matrix-free insulator
// panel of 16 complex64 columns, the steps n >= 3 run two at a time
// (stencil2_applies / launch_stencil2 in stencil_step.cu).
void filter_panel(const Matrix& M, double alpha, double beta, const double* gc, int Np, char* X,
                  int64_t ld, int nb, chebfd_dtype dt, double* moments, int64_t mom_ld,
                  char* U, char* W, int64_t ldw, double* partials, unsigned int* counter,
                  cudaStream_t s, char* W2 = nullptr, char* W3 = nullptr);
bool stencil2_applies(const Matrix& M, chebfd_dtype dt, int nb);
void launch_stencil2(const Matrix& M, const void* u0, const void* um, void* u1, void* u2,
                     void* y, int64_t ldw, int64_t ldy, double alpha, double beta, double c1,
                     double c2, cudaStream_t s);

void launch_random_block(void* X, int64_t n, int64_t ld, int nb, int col0, int ns_total,
                         uint64_t seed, chebfd_dtype dt, cudaStream_t stream);
void launch_kpm_probes(void* X, int64_t n, int64_t ld, int R, uint64_t seed, chebfd_dtype dt,
                       cudaStream_t stream);

// Device SplitMix64: i-th output of the generator started at seed*256 + stream.
__host__ __device__ inline uint64_t splitmix_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t splitmix_word(uint64_t seed, uint64_t stream,
                                                  uint64_t index) {
    uint64_t state = seed * 256ULL + stream;
    return splitmix_mix(state + (index + 1ULL) * 0x9E3779B97F4A7C15ULL);
}
__host__ __device__ inline double splitmix_uniform(uint64_t seed, uint64_t stream,
                                                   uint64_t index) {
    return (double)(splitmix_word(seed, stream, index) >> 11) * 0x1.0p-53;
}

constexpr uint64_t STREAM_DISORDER = 0;
constexpr uint64_t STREAM_SEARCH = 1;
constexpr uint64_t STREAM_KPM = 2;
constexpr uint64_t STREAM_REFILL = 3;
constexpr uint64_t STREAM_LANCZOS = 4;

}  // namespace chebfd

struct chebfd_matrix {
    chebfd::Matrix m;
};
