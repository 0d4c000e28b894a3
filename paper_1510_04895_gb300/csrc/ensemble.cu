// Ensembles of independent matrices (disorder realisations) filtered together.
//
// The instances are stored as one block-diagonal SELL matrix (instance i owns
// rows [off_i, off_i + N_i) and their columns), the search blocks of all
// instances as one row-major block with the same n_b.  One launch of the
// fused Chebyshev step then advances every instance by one step; each row
// reads its instance's alpha, beta and g_n c_n from a small coefficient table.
// The N_p launches of a filter are captured once into a CUDA graph and
// replayed, so a whole ensemble filter is one graph launch.  A host-side
// autotuner picks the SELL chunk height, the panel width and the row tile by
// timing a few steps of each candidate.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace chebfd {

int max_panel_width(chebfd_dtype dt);
void validate_block(const Matrix& M, chebfd_dtype dt, const void* X, int64_t ld, int nb);

namespace {

int grid_for(int64_t work) {
    return (int)std::min<int64_t>(std::max<int64_t>((work + 255) / 256, 1), 16384);
}

// Copy instance rows into the ensemble layout (uniform width L, chunk height C).
template <bool CPLX>
__global__ void ens_fill_uniform(const int32_t* col, const double* v64, const float* v32,
                                 int64_t n_i, int L, int64_t row_off, int C, int32_t* dcol,
                                 double* d64, float* d32) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_i * L;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / L;
        const int j = (int)(t - r * L);
        const int64_t R = row_off + r;
        const int64_t k = R / C;
        const int64_t dst = k * (int64_t)C * L + (int64_t)j * C + (R - k * C);
        const int64_t src = r * L + j;  // source chunk height 1
        dcol[dst] = col[src] + (int32_t)row_off;
        if (CPLX) {
            d64[2 * dst] = v64[2 * src];
            d64[2 * dst + 1] = v64[2 * src + 1];
            if (v32) {
                d32[2 * dst] = v32[2 * src];
                d32[2 * dst + 1] = v32[2 * src + 1];
            }
        } else {
            d64[dst] = v64[src];
            if (v32) d32[dst] = v32[src];
        }
    }
}

__global__ void ens_chunk_uniform(int64_t nchunks, int C, int L, int64_t* chunk_ptr,
                                  int32_t* chunk_len) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= nchunks;
         k += (int64_t)gridDim.x * blockDim.x) {
        chunk_ptr[k] = k * (int64_t)C * L;
        if (k < nchunks) chunk_len[k] = L;
    }
}

__global__ void ens_fill_bell_cols(const int32_t* in, int64_t count, int32_t shift, int32_t* out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        out[t] = in[t] + shift;
}

__global__ void fill_int_kernel(int32_t* p, int64_t n, int32_t v) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x)
        p[t] = v;
}

}  // namespace

}  // namespace chebfd

struct chebfd_ensemble {
    chebfd::Matrix m;                 // block-diagonal SELL (owned arrays)
    int count = 0;
    std::vector<int64_t> offsets;     // count + 1 row offsets
    int32_t* row_inst = nullptr;      // instance of each row
    double* coef = nullptr;           // [count][Np + 4]: alpha, beta, gc_0..gc_Np, beta/alpha
    int Np = 0;
    int panel = 0, tile = 0;          // tuned launch shape (0 = defaults)
    void* work = nullptr;             // U and W work vectors
    size_t work_bytes = 0;
    std::map<std::tuple<void*, int64_t, int, int, int, int, int>, cudaGraphExec_t> graphs;
};

namespace chebfd {

namespace {

void free_ensemble(chebfd_ensemble* E) {
    for (auto& kv : E->graphs) cudaGraphExecDestroy(kv.second);
    E->graphs.clear();
    cudaFree(E->m.chunk_ptr);
    cudaFree(E->m.chunk_len);
    cudaFree(E->m.col);
    cudaFree(E->m.val64);
    cudaFree(E->m.val32);
    cudaFree(E->m.bell_col);
    cudaFree(E->m.bell_val32);
    cudaFree(E->row_inst);
    cudaFree(E->coef);
    cudaFree(E->work);
}

void ensemble_build(chebfd_ensemble* E, const chebfd_matrix* const* Hs, int count, int C,
                    cudaStream_t s) {
    CHEBFD_REQUIRE(Hs && count >= 1, CHEBFD_EINVAL, "need at least one matrix");
    CHEBFD_REQUIRE(C >= 1 && C <= 32 && (C & (C - 1)) == 0, CHEBFD_EINVAL,
                   "chunk height must be a power of two in [1, 32]");
    const Matrix& M0 = Hs[0]->m;
    const bool cplx = M0.complex_values;
    bool single = true;
    const int L = M0.uniform_width;
    int64_t n = 0;
    E->offsets.assign(1, 0);
    for (int i = 0; i < count; ++i) {
        CHEBFD_REQUIRE(Hs[i] != nullptr, CHEBFD_EINVAL, "null matrix in ensemble");
        const Matrix& Mi = Hs[i]->m;
        CHEBFD_REQUIRE(Mi.complex_values == cplx, CHEBFD_EINVAL,
                       "ensemble members must all be complex or all real");
        CHEBFD_REQUIRE(Mi.C == 1 && Mi.identity_perm, CHEBFD_EINVAL,
                       "ensemble members must be built with sell_C = 1, sell_sigma = 1");
        CHEBFD_REQUIRE(L > 0 && Mi.uniform_width == L, CHEBFD_EUNSUPPORTED,
                       "ensemble members must share one constant row width");
        CHEBFD_REQUIRE(Mi.n % C == 0, CHEBFD_EINVAL,
                       "every member dimension must be a multiple of the chunk height");
        single = single && Mi.val32 != nullptr;
        n += Mi.n;
        E->offsets.push_back(n);
    }
    CHEBFD_REQUIRE(n < (1LL << 31), CHEBFD_EINVAL, "ensemble dimension must be < 2^31");
    Matrix& M = E->m;
    M = Matrix{};
    M.n = n;
    M.complex_values = cplx;
    M.identity_perm = true;
    M.C = C;
    M.sigma = 1;
    M.nchunks = n / C;
    M.max_row_len = L;
    M.uniform_width = L;
    M.nnz = n * L;
    M.nnz_padded = n * L;
    M.device = M0.device;
    M.num_sms = M0.num_sms;
    const size_t vs = cplx ? 16 : 8;
    CHEBFD_CHECK_CUDA(cudaMalloc(&M.chunk_ptr, (M.nchunks + 1) * sizeof(int64_t)));
    CHEBFD_CHECK_CUDA(cudaMalloc(&M.chunk_len, M.nchunks * sizeof(int32_t)));
    CHEBFD_CHECK_CUDA(cudaMalloc(&M.col, M.nnz_padded * sizeof(int32_t)));
    CHEBFD_CHECK_CUDA(cudaMalloc(&M.val64, M.nnz_padded * vs));
    if (single) CHEBFD_CHECK_CUDA(cudaMalloc(&M.val32, M.nnz_padded * vs / 2));
    CHEBFD_CHECK_CUDA(cudaMalloc(&E->row_inst, n * sizeof(int32_t)));
    ens_chunk_uniform<<<grid_for(M.nchunks + 1), 256, 0, s>>>(M.nchunks, C, L, M.chunk_ptr,
                                                              M.chunk_len);
    for (int i = 0; i < count; ++i) {
        const Matrix& Mi = Hs[i]->m;
        const int64_t off = E->offsets[i];
        if (cplx)
            ens_fill_uniform<true><<<grid_for(Mi.n * L), 256, 0, s>>>(
                Mi.col, (const double*)Mi.val64, single ? (const float*)Mi.val32 : nullptr, Mi.n,
                L, off, C, M.col, (double*)M.val64, (float*)M.val32);
        else
            ens_fill_uniform<false><<<grid_for(Mi.n * L), 256, 0, s>>>(
                Mi.col, (const double*)Mi.val64, single ? (const float*)Mi.val32 : nullptr, Mi.n,
                L, off, C, M.col, (double*)M.val64, (float*)M.val32);
        fill_int_kernel<<<grid_for(Mi.n), 256, 0, s>>>(E->row_inst + off, Mi.n, i);
    }
    // blocked copy: the members' blocked copies one after the other, block
    // columns shifted by the member's first block row (offsets are multiples
    // of 4: every member dimension is)
    bool blocked = single && cplx;
    for (int i = 0; i < count && blocked; ++i)
        blocked = Hs[i]->m.bell_col != nullptr && Hs[i]->m.n % kBellB == 0;
    if (blocked) {
        const int64_t nbr = n / kBellB;
        const size_t vb = (size_t)kBellLB * kBellB * kBellB * sizeof(float2);
        CHEBFD_CHECK_CUDA(cudaMalloc(&M.bell_col, nbr * kBellLB * sizeof(int32_t)));
        CHEBFD_CHECK_CUDA(cudaMalloc(&M.bell_val32, nbr * vb));
        for (int i = 0; i < count; ++i) {
            const Matrix& Mi = Hs[i]->m;
            const int64_t b0 = E->offsets[i] / kBellB, nbi = Mi.n / kBellB;
            ens_fill_bell_cols<<<grid_for(nbi * kBellLB), 256, 0, s>>>(
                Mi.bell_col, nbi * kBellLB, (int32_t)b0, M.bell_col + b0 * kBellLB);
            CHEBFD_CHECK_CUDA(cudaMemcpyAsync((char*)M.bell_val32 + b0 * vb, Mi.bell_val32,
                                              nbi * vb, cudaMemcpyDeviceToDevice, s));
        }
        M.bell_enabled = true;
    }
    CHEBFD_CHECK_CUDA(cudaGetLastError());
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
    E->count = count;
}

void set_coeffs(chebfd_ensemble* E, const double* alpha, const double* beta, const double* gc,
                int Np, cudaStream_t s) {
    CHEBFD_REQUIRE(alpha && beta && gc && Np >= 2, CHEBFD_EINVAL, "bad coefficient arguments");
    const int ldc = Np + 4;
    std::vector<double> h((size_t)E->count * ldc);
    for (int i = 0; i < E->count; ++i) {
        h[(size_t)i * ldc] = alpha[i];
        h[(size_t)i * ldc + 1] = beta[i];
        for (int n = 0; n <= Np; ++n) h[(size_t)i * ldc + 2 + n] = gc[(size_t)i * (Np + 1) + n];
        h[(size_t)i * ldc + Np + 3] = beta[i] / alpha[i];  // diagonal shift of the blocked step
    }
    if (Np != E->Np) {
        for (auto& kv : E->graphs) cudaGraphExecDestroy(kv.second);
        E->graphs.clear();
        cudaFree(E->coef);
        E->coef = nullptr;
        CHEBFD_CHECK_CUDA(cudaMalloc(&E->coef, h.size() * sizeof(double)));
        E->Np = Np;
    }
    CHEBFD_CHECK_CUDA(
        cudaMemcpyAsync(E->coef, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
}

int64_t padded_cols(chebfd_dtype dt, int nb) {
    const int64_t per = (int64_t)(16 / dtype_size(dt));
    return ((nb + per - 1) / per) * per;
}

// Queue the whole ensemble filter (all panels, all N_p steps) on stream s.
void queue_filter(chebfd_ensemble* E, void* X, int64_t ld, int nb, chebfd_dtype dt,
                  cudaStream_t s) {
    const Matrix& M = E->m;
    const int pw = E->panel > 0 ? std::min(E->panel, max_panel_width(dt)) : max_panel_width(dt);
    const int wmax = std::min(pw, nb);
    const int64_t ldw = padded_cols(dt, wmax);
    const size_t es = dtype_size(dt);
    char* U = (char*)E->work;
    char* W = U + (size_t)M.n * ldw * es;
    const int Np = E->Np;
    for (int p0 = 0; p0 < nb; p0 += pw) {
        const int pnb = std::min(pw, nb - p0);
        CHEBFD_REQUIRE(((size_t)pnb * es) % 16 == 0, CHEBFD_EINVAL,
                       "panel width * element size must be a multiple of 16 bytes");
        char* Xp = (char*)X + p0 * es;
        StepArgs a{};
        a.nb = pnb;
        a.tile = E->tile;
        a.coef = E->coef;
        a.row_inst = E->row_inst;
        a.coef_ld = Np + 4;
        a.gather = Xp;
        a.ldg = ld;
        a.w = U;
        a.ldw = ldw;
        a.mom_step = 1;
        launch_step(M, dt, MODE_SPMV, a, s);
        a.gather = U;
        a.ldg = ldw;
        a.w = W;
        a.y = Xp;
        a.ldy = ld;
        a.mom_step = 2;
        launch_step(M, dt, MODE_SECOND, a, s);
        char* u = U;
        char* w = W;
        for (int n = 3; n <= Np; ++n) {
            std::swap(u, w);
            a.gather = u;
            a.w = w;
            a.mom_step = n;
            launch_step(M, dt, MODE_STEP, a, s);
        }
    }
}

void ensure_work(chebfd_ensemble* E, int nb, chebfd_dtype dt) {
    const int pw = E->panel > 0 ? std::min(E->panel, max_panel_width(dt)) : max_panel_width(dt);
    const size_t need = 2 * (size_t)E->m.n * padded_cols(dt, std::min(pw, nb)) * dtype_size(dt);
    if (need <= E->work_bytes) return;
    for (auto& kv : E->graphs) cudaGraphExecDestroy(kv.second);
    E->graphs.clear();
    cudaFree(E->work);
    E->work = nullptr;
    E->work_bytes = 0;
    CHEBFD_CHECK_CUDA(cudaMalloc(&E->work, need));
    E->work_bytes = need;
}

void ensemble_filter(chebfd_ensemble* E, void* X, int64_t ld, int nb, chebfd_dtype dt,
                     bool use_graph, cudaStream_t s) {
    validate_block(E->m, dt, X, ld, nb);
    CHEBFD_REQUIRE(E->coef != nullptr, CHEBFD_EINVAL, "set the ensemble coefficients first");
    ensure_work(E, nb, dt);
    if (!use_graph) {
        queue_filter(E, X, ld, nb, dt, s);
        return;
    }
    const auto key = std::make_tuple(X, ld, nb, (int)dt, E->Np, E->panel, E->tile);
    auto it = E->graphs.find(key);
    if (it == E->graphs.end()) {
        cudaStream_t cs;
        CHEBFD_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        CHEBFD_CHECK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        try {
            queue_filter(E, X, ld, nb, dt, cs);
        } catch (...) {
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            throw;
        }
        CHEBFD_CHECK_CUDA(cudaStreamEndCapture(cs, &g));
        cudaStreamDestroy(cs);
        const cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        CHEBFD_CHECK_CUDA(e);
        it = E->graphs.emplace(key, ge).first;
    }
    CHEBFD_CHECK_CUDA(cudaGraphLaunch(it->second, s));
}

double time_steps(chebfd_ensemble* E, void* X, int64_t ld, int nb, chebfd_dtype dt,
                  cudaStream_t s) {
    cudaEvent_t e0, e1;
    CHEBFD_CHECK_CUDA(cudaEventCreate(&e0));
    CHEBFD_CHECK_CUDA(cudaEventCreate(&e1));
    ensemble_filter(E, X, ld, nb, dt, false, s);  // warm-up
    CHEBFD_CHECK_CUDA(cudaEventRecord(e0, s));
    ensemble_filter(E, X, ld, nb, dt, false, s);
    CHEBFD_CHECK_CUDA(cudaEventRecord(e1, s));
    CHEBFD_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

}  // namespace

void orthonormalize_impl(void* Yv, int64_t n, int ns, int64_t ld, chebfd_dtype dt,
                         uint64_t seed, int64_t* refill_counter, int* rank_out, cudaStream_t s);
void rayleigh_ritz_impl(const Matrix& M, void* Yv, int64_t ld, int ns, chebfd_dtype dt,
                        double* theta_host, double* res_host, void* HY_out, cudaStream_t s);
void convert_block_impl(const void* X, chebfd_dtype xdt, int64_t ldx, void* Y, chebfd_dtype ydt,
                        int64_t ldy, int64_t n, int nb, cudaStream_t s);
void launch_random_block(void* X, int64_t n, int64_t ld, int nb, int col0, int ns_total,
                         uint64_t seed, chebfd_dtype dt, cudaStream_t stream);
void fill_result(chebfd_result* R, const std::vector<int>& acc, const std::vector<double>& theta,
                 const std::vector<double>& res, const void* Y, int64_t n, int64_t ld,
                 size_t es, int iterations, bool converged, int fp64_its, int64_t n_mvm,
                 double a, double b, cudaStream_t s);
chebfd_result* new_result();
void set_iterations(chebfd_result* R, const std::vector<chebfd_iteration_info>& recs);

// The ChebFD iteration of Sec. 3.1 for every member of an ensemble at once:
// one ensemble filter per iteration (all members, one graph launch), then
// SVQB and Rayleigh-Ritz member by member on their row slices, with the
// convergence and ghost test of chebfd_solve per member.  A converged
// member's pairs are taken at that iteration; its rows keep being filtered
// (the launch covers all rows) but are no longer projected.  MIXED precision
// runs the ensemble filter in single precision until every unconverged
// member has stalled above 1e-9 ||H_i|| (largest accepted residual falling
// less than 2x), then in FP64.
void solve_batched_impl(chebfd_ensemble* E, const chebfd_matrix* const* Hs, const double* av,
                        const double* bv, const chebfd_params& p0, cudaStream_t s,
                        chebfd_result** outs, int* iterations_out) {
    chebfd_params p = p0;
    CHEBFD_REQUIRE(p.ns >= 4 && p.ns <= 1024 && p.ns % 4 == 0, CHEBFD_EINVAL,
                   "need 4 <= ns <= 1024, ns a multiple of 4");
    CHEBFD_REQUIRE(p.Np >= 2 && p.lam_hi > p.lam_lo && p.eps > 0.0, CHEBFD_EINVAL,
                   "bad solve parameters");
    if (p.mu <= 0.0) p.mu = 2.0;
    if (p.max_iter <= 0) p.max_iter = 50;
    const int count = E->count;
    const bool cplx = E->m.complex_values;
    const chebfd_dtype d64 = cplx ? CHEBFD_C128 : CHEBFD_R64;
    const chebfd_dtype d32 = cplx ? CHEBFD_C64 : CHEBFD_R32;
    CHEBFD_REQUIRE(p.flags == 0, CHEBFD_EUNSUPPORTED, "batched solve takes no solve flags");
    CHEBFD_REQUIRE(p.precision == CHEBFD_PRECISION_FP64 || p.precision == CHEBFD_PRECISION_MIXED,
                   CHEBFD_EUNSUPPORTED, "batched solve runs FP64 or MIXED precision");
    const bool mixed = p.precision == CHEBFD_PRECISION_MIXED;
    CHEBFD_REQUIRE(!mixed || E->m.val32 != nullptr, CHEBFD_EINVAL,
                   "mixed precision needs members built with also_single");
    for (int i = 0; i < count; ++i) {
        CHEBFD_REQUIRE(Hs[i] && Hs[i]->m.n == E->offsets[i + 1] - E->offsets[i], CHEBFD_EINVAL,
                       "member matrices do not match the ensemble");
        CHEBFD_REQUIRE(bv[i] > av[i], CHEBFD_EINVAL, "need b > a for every member");
        outs[i] = nullptr;
    }
    // per-member coefficients of the common window (narrowed by window_inset)
    CHEBFD_REQUIRE(p.window_inset >= 0.0 && p.window_inset < 1.0, CHEBFD_EINVAL,
                   "need 0 <= window_inset < 1");
    const double wc = 0.5 * (p.lam_lo + p.lam_hi),
                 wh = 0.5 * (p.lam_hi - p.lam_lo) * (1.0 - p.window_inset);
    std::vector<double> al(count), be(count), gc((size_t)count * (p.Np + 1));
    for (int i = 0; i < count; ++i) {
        al[i] = 2.0 / (bv[i] - av[i]);
        be[i] = (av[i] + bv[i]) / (av[i] - bv[i]);
        const chebfd_status st = chebfd_window_coeffs(av[i], bv[i], wc - wh, wc + wh, p.Np,
                                                      (chebfd_kernel)p.kernel, p.mu,
                                                      gc.data() + (size_t)i * (p.Np + 1));
        CHEBFD_REQUIRE(st == CHEBFD_OK, st, "coefficient construction failed");
    }
    set_coeffs(E, al.data(), be.data(), gc.data(), p.Np, s);
    const int64_t n = E->m.n;
    const int ns = p.ns;
    const int64_t ld = ns;
    void *Y64 = nullptr, *X32 = nullptr;
    auto cleanup = [&]() {
        cudaFree(Y64);
        cudaFree(X32);
    };
    try {
        CHEBFD_CHECK_CUDA(cudaMalloc(&Y64, (size_t)n * ld * dtype_size(d64)));
        if (mixed) CHEBFD_CHECK_CUDA(cudaMalloc(&X32, (size_t)n * ld * dtype_size(d32)));
        launch_random_block(Y64, n, ld, ns, 0, ns, p.seed, d64, s);
        bool single_phase = mixed;
        if (mixed) convert_block_impl(Y64, d64, ld, X32, d32, ld, n, ns, s);
        struct State {
            bool done = false, stalled = false, prev_empty = false;
            double prev_worst = -1.0;
            std::vector<double> prev_theta, prev_res;
            std::vector<chebfd_iteration_info> recs;
            int64_t refill = 0;
        };
        std::vector<State> st(count);
        std::vector<double> theta(ns), res(ns);
        int it = 0, fp64_its = 0, remaining = count;
        for (it = 1; it <= p.max_iter && remaining > 0; ++it) {
            if (single_phase) {
                ensemble_filter(E, X32, ld, ns, d32, true, s);
                convert_block_impl(X32, d32, ld, Y64, d64, ld, n, ns, s);
            } else {
                ensemble_filter(E, Y64, ld, ns, d64, true, s);
                ++fp64_its;
            }
            bool all_stalled = true;
            for (int i = 0; i < count; ++i) {
                State& S = st[i];
                if (S.done) continue;
                const Matrix& Mi = Hs[i]->m;
                void* Yi = (char*)Y64 + (size_t)E->offsets[i] * ld * dtype_size(d64);
                orthonormalize_impl(Yi, Mi.n, ns, ld, d64, p.seed + 1000003ULL * i, &S.refill,
                                    nullptr, s);
                rayleigh_ritz_impl(Mi, Yi, ld, ns, d64, theta.data(), res.data(), nullptr, s);
                const double normH = std::max(std::fabs(av[i]), std::fabs(bv[i]));
                std::vector<int> acc;
                int in_window = 0, live = 0;
                for (int k = 0; k < ns; ++k) {
                    if (!(theta[k] >= p.lam_lo && theta[k] <= p.lam_hi)) continue;
                    ++in_window;
                    bool ghost = false, falling = false;
                    if (!S.prev_theta.empty()) {
                        int j = 0;
                        for (int q = 1; q < ns; ++q)
                            if (std::fabs(S.prev_theta[q] - theta[k]) <
                                std::fabs(S.prev_theta[j] - theta[k]))
                                j = q;
                        ghost = res[k] > std::sqrt(p.eps) * normH &&
                                !(S.prev_res[j] >= 10.0 * res[k]);
                        falling = res[k] <= 0.9 * S.prev_res[j];
                    }
                    if (!ghost) acc.push_back(k);
                    if (!ghost || falling) ++live;
                }
                double worst = 0.0, best = -1.0;
                chebfd_iteration_info rec{};
                rec.iteration = it;
                rec.fp64_filter = single_phase ? 0 : 1;
                for (int k : acc) {
                    worst = std::max(worst, res[k]);
                    best = best < 0.0 ? res[k] : std::min(best, res[k]);
                    if (res[k] <= p.eps * normH) ++rec.converged_pairs;
                }
                rec.in_window = in_window;
                rec.accepted = (int)acc.size();
                rec.ghosts = in_window - rec.accepted;
                rec.res_min = best;
                rec.res_max = acc.empty() ? -1.0 : worst;
                S.recs.push_back(rec);
                bool conv = !acc.empty() && worst <= p.eps * normH;
                // empty window: two successive iterations (from the second on)
                // without an in-window pair that is accepted or still converging
                const bool empty_now = !S.prev_theta.empty() && live == 0;
                const bool empty = empty_now && S.prev_empty;
                S.prev_empty = empty_now;
                if (empty || (conv && !single_phase)) {
                    outs[i] = new_result();
                    fill_result(outs[i], acc, theta, res, Yi, Mi.n, ld, dtype_size(d64), it, true,
                                fp64_its, (int64_t)it * ns * p.Np, av[i], bv[i], s);
                    set_iterations(outs[i], S.recs);
                    S.done = true;
                    --remaining;
                    continue;
                }
                if (single_phase) {
                    S.stalled = S.stalled || conv ||
                                (S.prev_worst > 0.0 && worst > 1e-9 * normH &&
                                 worst > 0.5 * S.prev_worst);
                    all_stalled = all_stalled && S.stalled;
                }
                S.prev_worst = worst;
                S.prev_theta = theta;
                S.prev_res = res;
                if (it == p.max_iter) {
                    outs[i] = new_result();
                    fill_result(outs[i], acc, theta, res, Yi, Mi.n, ld, dtype_size(d64), it,
                                false, fp64_its, (int64_t)it * ns * p.Np, av[i], bv[i], s);
                    set_iterations(outs[i], S.recs);
                }
            }
            if (single_phase && all_stalled) single_phase = false;
            if (single_phase) convert_block_impl(Y64, d64, ld, X32, d32, ld, n, ns, s);
        }
        for (int i = 0; i < count; ++i)
            if (!outs[i]) {  // iteration budget ended before this member was visited
                outs[i] = new_result();
                fill_result(outs[i], {}, theta, res, Y64, Hs[i]->m.n, ld, dtype_size(d64), it,
                            false, fp64_its, (int64_t)it * ns * p.Np, av[i], bv[i], s);
            }
        if (iterations_out) *iterations_out = std::min(it, p.max_iter);
    } catch (...) {
        cleanup();
        for (int i = 0; i < count; ++i)
            if (outs[i]) {
                chebfd_result_destroy(outs[i]);
                outs[i] = nullptr;
            }
        throw;
    }
    cleanup();
}

}  // namespace chebfd

using namespace chebfd;

extern "C" {

chebfd_status chebfd_ensemble_create(const chebfd_matrix* const* Hs, int count, int sell_C,
                                     void* stream, chebfd_ensemble** out) {
    chebfd_ensemble* E = nullptr;
    chebfd_status st = guarded([&] {
        CHEBFD_REQUIRE(out, CHEBFD_EINVAL, "null output");
        E = new chebfd_ensemble();
        ensemble_build(E, Hs, count, sell_C, as_stream(stream));
    });
    if (st != CHEBFD_OK) {
        if (E) {
            free_ensemble(E);
            delete E;
        }
        return st;
    }
    *out = E;
    return CHEBFD_OK;
}

chebfd_status chebfd_ensemble_info(const chebfd_ensemble* E, int64_t* n_total, int* count,
                                   int64_t* row_offsets, int* sell_C, int* panel, int* tile) {
    return guarded([&] {
        CHEBFD_REQUIRE(E, CHEBFD_EINVAL, "null ensemble");
        if (n_total) *n_total = E->m.n;
        if (count) *count = E->count;
        if (row_offsets) std::copy(E->offsets.begin(), E->offsets.end(), row_offsets);
        if (sell_C) *sell_C = E->m.C;
        if (panel) *panel = E->panel;
        if (tile) *tile = E->tile;
    });
}

chebfd_status chebfd_ensemble_set_coeffs(chebfd_ensemble* E, const double* alpha,
                                         const double* beta, const double* gc, int Np,
                                         void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(E, CHEBFD_EINVAL, "null ensemble");
        set_coeffs(E, alpha, beta, gc, Np, as_stream(stream));
    });
}

chebfd_status chebfd_ensemble_set_launch(chebfd_ensemble* E, int panel, int tile) {
    return guarded([&] {
        CHEBFD_REQUIRE(E && panel >= 0 && tile >= 0, CHEBFD_EINVAL, "bad launch shape");
        E->panel = panel;
        E->tile = tile;
    });
}

chebfd_status chebfd_ensemble_filter(chebfd_ensemble* E, void* X, int64_t ld, int nb,
                                     chebfd_dtype vdt, int use_graph, void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(E, CHEBFD_EINVAL, "null ensemble");
        ensemble_filter(E, X, ld, nb, vdt, use_graph != 0, as_stream(stream));
    });
}

chebfd_status chebfd_ensemble_autotune(const chebfd_matrix* const* Hs, int count, void* X,
                                       int64_t ld, int nb, chebfd_dtype vdt, void* stream,
                                       chebfd_ensemble** out, double* best_ms) {
    chebfd_ensemble* best = nullptr;
    chebfd_status st = guarded([&] {
        CHEBFD_REQUIRE(out && X, CHEBFD_EINVAL, "null argument");
        cudaStream_t s = as_stream(stream);
        // candidate shapes: SELL chunk height C, panel width, row tile
        const int Cs[] = {1, 2, 4};
        const int tiles[] = {1, 4, 16};
        std::vector<int> panels;
        for (int p : {16, 32, 48, 64, 128})
            if (p <= max_panel_width(vdt) && ((size_t)p * dtype_size(vdt)) % 16 == 0 && p <= nb)
                panels.push_back(p);
        if (panels.empty()) panels.push_back(std::min(nb, max_panel_width(vdt)));
        std::vector<double> al(count, 0.1), be(count, 0.0), gc((size_t)count * 8, 0.0);
        double best_t = 1e30;
        int best_panel = 0, best_tile = 0;
        for (int C : Cs) {
            bool ok = true;
            for (int i = 0; i < count; ++i) ok = ok && Hs[i] && Hs[i]->m.n % C == 0;
            if (!ok) continue;
            auto* E = new chebfd_ensemble();
            try {
                ensemble_build(E, Hs, count, C, s);
                set_coeffs(E, al.data(), be.data(), gc.data(), 7, s);
                for (int p : panels)
                    for (int t : tiles) {
                        E->panel = p;
                        E->tile = t;
                        const double ms = time_steps(E, X, ld, nb, vdt, s);
                        if (ms < best_t) {
                            best_t = ms;
                            best_panel = p;
                            best_tile = t;
                            if (best != E) {
                                if (best) {
                                    free_ensemble(best);
                                    delete best;
                                }
                                best = E;
                            }
                        }
                    }
            } catch (...) {
                if (E != best) {
                    free_ensemble(E);
                    delete E;
                }
                throw;
            }
            if (E != best) {
                free_ensemble(E);
                delete E;
            }
        }
        CHEBFD_REQUIRE(best != nullptr, CHEBFD_EINVAL, "no admissible ensemble layout");
        best->panel = best_panel;
        best->tile = best_tile;
        for (auto& kv : best->graphs) cudaGraphExecDestroy(kv.second);
        best->graphs.clear();
        if (best_ms) *best_ms = best_t / 7.0;  // per Chebyshev step (7 launches per panel set)
    });
    if (st != CHEBFD_OK) {
        if (best) {
            free_ensemble(best);
            delete best;
        }
        return st;
    }
    *out = best;
    return CHEBFD_OK;
}

chebfd_status chebfd_solve_batched(chebfd_ensemble* E, const chebfd_matrix* const* Hs,
                                   const double* a, const double* b, const chebfd_params* p,
                                   void* stream, chebfd_result** outs, int* iterations) {
    return guarded([&] {
        CHEBFD_REQUIRE(E && Hs && a && b && p && outs, CHEBFD_EINVAL, "null argument");
        solve_batched_impl(E, Hs, a, b, *p, as_stream(stream), outs, iterations);
    });
}

chebfd_status chebfd_ensemble_destroy(chebfd_ensemble* E) {
    return guarded([&] {
        if (!E) return;
        free_ensemble(E);
        delete E;
    });
}

}  // extern "C"
