// The ChebFD iteration (Sec. 3.1, steps 4-8) orchestrated on the host around
// the device kernels: filter, SVQB, Rayleigh-Ritz, convergence and ghost test.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace chebfd {

void filter_block_df_impl(const Matrix& M, double alpha, double beta, const double* gc, int Np,
                          void* X, int64_t ld, int nb, cudaStream_t s);
void ortho_rr_impl(const Matrix& M, void* Yv, int64_t ld, int ns, chebfd_dtype dt, uint64_t seed,
                   int64_t* refill_counter, double* theta_host, double* res_host, bool df,
                   bool harmonic, double tau, cudaStream_t s, double* phase_seconds);
void harmonic_ritz_impl(const Matrix& M, void* Yv, int64_t ld, int ns, chebfd_dtype dt, double tau,
                        double* theta_host, double* res_host, cudaStream_t s);

void filter_block_impl(const Matrix& M, double alpha, double beta, const double* gc, int Np,
                       void* X, int64_t ld, int nb, chebfd_dtype dt, double* moments,
                       cudaStream_t s, int panel = 0);
void scale_bounds_impl(const Matrix& M, int steps, uint64_t seed, double* a_out, double* b_out,
                       cudaStream_t s);
void orthonormalize_impl(void* Yv, int64_t n, int ns, int64_t ld, chebfd_dtype dt,
                         uint64_t seed, int64_t* refill_counter, int* rank_out, cudaStream_t s);
void rayleigh_ritz_impl(const Matrix& M, void* Yv, int64_t ld, int ns, chebfd_dtype dt,
                        double* theta_host, double* res_host, void* HY_out, cudaStream_t s);
void convert_block_impl(const void* X, chebfd_dtype xdt, int64_t ldx, void* Y, chebfd_dtype ydt,
                        int64_t ldy, int64_t n, int nb, cudaStream_t s);
void launch_random_block(void* X, int64_t n, int64_t ld, int nb, int col0, int ns_total,
                         uint64_t seed, chebfd_dtype dt, cudaStream_t stream);
int max_panel_width(chebfd_dtype dt);
int adaptive_degree(const std::vector<double>& mu, int64_t N, double a, double b, double lo,
                    double hi, int ns, int Np0, double* n_target, double* dprime);
void deflate_impl(bool cplx, const double* L, int nl, double* Y, int w, int64_t n, int64_t ld,
                  bool tensor, int sms, cudaStream_t s);
void gather_columns_impl(const double* src, int64_t ld, int64_t n, const std::vector<int>& idx,
                         bool cplx, double* dst, int64_t ldd, cudaStream_t s);

}  // namespace chebfd

struct chebfd_result;

namespace chebfd {
void fill_result(chebfd_result* R, const std::vector<int>& acc, const std::vector<double>& theta,
                 const std::vector<double>& res, const void* Y, int64_t n, int64_t ld,
                 size_t es, int iterations, bool converged, int fp64_its, int64_t n_mvm,
                 double a, double b, cudaStream_t s);
}  // namespace chebfd

struct chebfd_result {
    chebfd_result_info info{};
    std::vector<chebfd_iteration_info> iterations;
    std::vector<double> lambda, res;
    void* V = nullptr;
    int64_t n = 0;
    size_t elem_size = 0;
};

namespace chebfd {

namespace {

// gc[n] = g_n c_n (Sec. 2.1, Tab. Kernel) - the same construction as the
// chebfd_window_coeffs entry point.
std::vector<double> coefficients(double a, double b, double lo, double hi, int Np, int kernel,
                                 double mu) {
    std::vector<double> gc(Np + 1);
    const chebfd_status st =
        chebfd_window_coeffs(a, b, lo, hi, Np, (chebfd_kernel)kernel, mu, gc.data());
    CHEBFD_REQUIRE(st == CHEBFD_OK, st, "coefficient construction failed");
    return gc;
}

struct DevMem {
    void* p = nullptr;
    explicit DevMem(size_t bytes) {
        if (bytes) CHEBFD_CHECK_CUDA(cudaMalloc(&p, bytes));
    }
    ~DevMem() { cudaFree(p); }
    DevMem(const DevMem&) = delete;
    DevMem& operator=(const DevMem&) = delete;
};

double now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace

void solve_impl(const Matrix& M, const chebfd_params& p0, cudaStream_t s, chebfd_result* R) {
    chebfd_params p = p0;
    CHEBFD_REQUIRE(p.ns >= 4 && p.ns <= 1024 && p.ns % 4 == 0, CHEBFD_EINVAL,
                   "need 4 <= ns <= 1024, ns a multiple of 4");
    CHEBFD_REQUIRE(p.Np >= 2, CHEBFD_EINVAL, "need Np >= 2");
    CHEBFD_REQUIRE(p.lam_hi > p.lam_lo, CHEBFD_EINVAL, "need lam_hi > lam_lo");
    CHEBFD_REQUIRE(p.eps > 0.0, CHEBFD_EINVAL, "need eps > 0");
    CHEBFD_REQUIRE(p.window_inset >= 0.0 && p.window_inset < 1.0, CHEBFD_EINVAL,
                   "need 0 <= window_inset < 1");
    if (p.mu <= 0.0) p.mu = 2.0;
    if (p.max_iter <= 0) p.max_iter = 50;
    if (p.lanczos_steps <= 0) p.lanczos_steps = 30;
    const bool cplx = M.complex_values;
    const chebfd_dtype d64 = cplx ? CHEBFD_C128 : CHEBFD_R64;
    const chebfd_dtype d32 = cplx ? CHEBFD_C64 : CHEBFD_R32;
    CHEBFD_REQUIRE(p.precision >= CHEBFD_PRECISION_FP64 &&
                       p.precision <= CHEBFD_PRECISION_MIXED_DF,
                   CHEBFD_EINVAL, "unknown precision");
    CHEBFD_REQUIRE((p.flags & ~(CHEBFD_SOLVE_HARMONIC | CHEBFD_SOLVE_ADAPTIVE |
                                CHEBFD_SOLVE_LOCKING)) == 0,
                   CHEBFD_EINVAL, "unknown solve flags");
    const bool harmonic = (p.flags & CHEBFD_SOLVE_HARMONIC) != 0;
    const bool adaptive = (p.flags & CHEBFD_SOLVE_ADAPTIVE) != 0;
    const bool locking = (p.flags & CHEBFD_SOLVE_LOCKING) != 0;
    CHEBFD_REQUIRE(!(locking && harmonic), CHEBFD_EINVAL,
                   "locking needs orthonormal Ritz vectors: not with harmonic pairs");
    const double tau = 0.5 * (p.lam_lo + p.lam_hi);
    const bool df = p.precision == CHEBFD_PRECISION_MIXED_DF;
    const bool mixed = p.precision == CHEBFD_PRECISION_MIXED || df;
    CHEBFD_REQUIRE(!mixed || M.val32 != nullptr, CHEBFD_EINVAL,
                   "mixed precision needs a matrix built with also_single");
    if (p.nb <= 0) p.nb = cplx ? 64 : 128;
    const double t_start = now();
    double a = p.a, b = p.b;
    if (!(b > a)) scale_bounds_impl(M, p.lanczos_steps, p.seed, &a, &b, s);
    const double normH = std::max(std::fabs(a), std::fabs(b));
    const double alpha = 2.0 / (b - a), beta = (a + b) / (a - b);
    // filter window: the target interval, narrowed by window_inset of its half-width
    const double wc = 0.5 * (p.lam_lo + p.lam_hi),
                 wh = 0.5 * (p.lam_hi - p.lam_lo) * (1.0 - p.window_inset);
    std::vector<double> gc = coefficients(a, b, wc - wh, wc + wh, p.Np, p.kernel, p.mu);
    int Np = p.Np;
    int64_t n_mvm = 0;
    const int64_t n = M.n;
    const int ns = p.ns;
    const int64_t ld = ns;  // rows start on 16 bytes in every precision (ns % 4 == 0)
    DevMem Y64((size_t)n * ld * dtype_size(d64));
    // locking: the locked vectors, and a second block for compacting the rest
    DevMem Lk(locking ? (size_t)n * ld * dtype_size(d64) : 0);
    DevMem Yb(locking ? (size_t)n * ld * dtype_size(d64) : 0);
    double* Y = (double*)Y64.p;
    double* Yalt = (double*)Yb.p;
    std::vector<double> lam_L, res_L;
    int nl = 0, nact = ns;
    DevMem X32(mixed ? (size_t)n * ld * dtype_size(d32) : 0);
    // moments of the first filter (adaptive degree): 2 Np x ns
    DevMem mom(adaptive ? (size_t)2 * p.Np * ns * sizeof(double) : 0);
    CHEBFD_CHECK_CUDA(cudaMemsetAsync(Y, 0, (size_t)n * ld * dtype_size(d64), s));
    launch_random_block(Y, n, ld, ns, 0, ns, p.seed, d64, s);
    bool single_phase = mixed;
    if (mixed) convert_block_impl(Y, d64, ld, X32.p, d32, ld, n, ns, s);

    std::vector<double> theta(ns), res(ns), prev_theta, prev_res;
    int64_t refill = 0;
    double prev_worst = -1.0;
    bool prev_empty = false;
    double t_filter = 0.0, t_dense = 0.0;
    int it = 0, fp64_its = 0;
    bool converged = false;
    std::vector<int> acc_idx;
    for (it = 1; it <= p.max_iter; ++it) {
        // ---- step 5: filter
        double t0 = now();
        const bool with_moments = adaptive && it == 1;
        double* mom_dev = with_moments ? (double*)mom.p : nullptr;
        const int Np_it = Np;
        if (single_phase) {
            filter_block_impl(M, alpha, beta, gc.data(), Np, X32.p, ld, nact, d32, mom_dev, s,
                              p.nb);
            convert_block_impl(X32.p, d32, ld, Y, d64, ld, n, nact, s);
        } else {
            if (df && !with_moments)
                filter_block_df_impl(M, alpha, beta, gc.data(), Np, Y, ld, nact, s);
            else
                filter_block_impl(M, alpha, beta, gc.data(), Np, Y, ld, nact, d64, mom_dev, s,
                                  p.nb);
            ++fp64_its;
        }
        // locking: the filtered block leaves the span of the locked vectors
        if (nl > 0) deflate_impl(cplx, (const double*)Lk.p, nl, Y, nact, n, ld, df, M.num_sms, s);
        CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
        n_mvm += (int64_t)nact * Np;
        if (with_moments) {
            // the n_s random columns as KPM probes: <x_k, T_n x_k> / <x_k, x_k>, averaged
            std::vector<double> h((size_t)2 * Np * ns), mu(2 * Np, 0.0);
            CHEBFD_CHECK_CUDA(cudaMemcpy(h.data(), mom.p, h.size() * sizeof(double),
                                         cudaMemcpyDeviceToHost));
            for (int k = 0; k < ns; ++k)
                for (int q = 0; q < 2 * Np; ++q) mu[q] += h[(size_t)q * ns + k] / h[k] / ns;
            Np = adaptive_degree(mu, n, a, b, p.lam_lo, p.lam_hi, ns, Np, nullptr, nullptr);
            gc = coefficients(a, b, wc - wh, wc + wh, Np, p.kernel, p.mu);
        }
        double t1 = now();
        t_filter += t1 - t0;
        chebfd_iteration_info rec{};
        rec.iteration = it;
        rec.Np = Np_it;
        rec.fp64_filter = single_phase ? 0 : 1;
        rec.seconds_filter = t1 - t0;
        // ---- steps 6-7: orthonormalise, Rayleigh-Ritz
        double phase[PH_COUNT] = {0, 0, 0, 0, 0, 0};
        const int64_t refill_before = refill;
        ortho_rr_impl(M, Y, ld, nact, d64, p.seed, &refill, theta.data(), res.data(), df,
                      harmonic, tau, s, phase);
        if (nl > 0 && refill != refill_before) {
            // refilled random columns: out of the locked span once more
            deflate_impl(cplx, (const double*)Lk.p, nl, Y, nact, n, ld, df, M.num_sms, s);
            orthonormalize_impl(Y, n, nact, ld, d64, p.seed, &refill, nullptr, s);
            rayleigh_ritz_impl(M, Y, ld, nact, d64, theta.data(), res.data(), nullptr, s);
        }
        rec.seconds_dense = now() - t1;
        t_dense += rec.seconds_dense;
        rec.seconds_gram = phase[PH_GRAM];
        rec.seconds_block_gemm = phase[PH_BLOCK_GEMM];
        rec.seconds_eigensolve = phase[PH_EIG];
        rec.seconds_hy = phase[PH_HY];
        rec.seconds_residuals = phase[PH_RESIDUAL];
        rec.seconds_other = phase[PH_OTHER];
        // ---- step 8: window membership, ghosts, convergence
        acc_idx.clear();
        int in_window = 0, live = 0;
        for (int k = 0; k < nact; ++k) {
            if (!(theta[k] >= p.lam_lo && theta[k] <= p.lam_hi)) continue;
            ++in_window;
            bool ghost = false, falling = false;
            if (!prev_theta.empty()) {
                int j = 0;
                for (int q = 1; q < (int)prev_theta.size(); ++q)
                    if (std::fabs(prev_theta[q] - theta[k]) < std::fabs(prev_theta[j] - theta[k]))
                        j = q;
                ghost = res[k] > std::sqrt(p.eps) * normH && !(prev_res[j] >= 10.0 * res[k]);
                falling = res[k] <= 0.9 * prev_res[j];
            }
            if (!ghost) acc_idx.push_back(k);
            if (!ghost || falling) ++live;
        }
        double worst = 0.0, best = -1.0;
        for (int k : acc_idx) {
            worst = std::max(worst, res[k]);
            best = best < 0.0 ? res[k] : std::min(best, res[k]);
            if (res[k] <= p.eps * normH) ++rec.converged_pairs;
        }
        rec.in_window = in_window;
        rec.accepted = (int)acc_idx.size();
        rec.ghosts = in_window - rec.accepted;
        rec.res_min = best;
        rec.res_max = acc_idx.empty() ? -1.0 : worst;
        rec.locked = nl;
        R->iterations.push_back(rec);
        converged = (!acc_idx.empty() || nl > 0) && worst <= p.eps * normH;
        // empty window: two successive iterations (from the second on) without
        // an in-window pair that is accepted or still converging (residual at
        // most 0.9 of the previous nearest pair's): the ghost-flagged pairs of a
        // weak filter keep converging, spurious in-window values stagnate
        const bool empty_now = !prev_theta.empty() && live == 0 && nl == 0;
        if (empty_now && prev_empty) {
            converged = true;
            break;
        }
        prev_empty = empty_now;
        if (converged && !single_phase) break;
        if (converged && single_phase) {
            // reached the target in single precision: confirm with one FP64 sweep
            single_phase = false;
        } else if (single_phase && prev_worst > 0.0 && worst > 1e-9 * normH &&
                   worst > 0.5 * prev_worst) {
            single_phase = false;  // residuals stalled at the single-precision floor
        }
        prev_worst = worst;
        // locking: converged accepted pairs, the smallest residuals first, four
        // at a time, leave the block (at least four columns stay)
        std::vector<int> keep;
        if (locking) {
            std::vector<int> done;
            for (int k : acc_idx)
                if (res[k] <= p.eps * normH) done.push_back(k);
            std::stable_sort(done.begin(), done.end(),
                             [&](int x, int y) { return res[x] < res[y]; });
            done.resize(done.size() / 4 * 4);
            if (!done.empty() && nact - (int)done.size() >= 4) {
                std::sort(done.begin(), done.end());
                const int ew = cplx ? 2 : 1;
                gather_columns_impl(Y, ld, n, done, cplx, (double*)Lk.p + (size_t)nl * ew, ld, s);
                for (int k : done) {
                    lam_L.push_back(theta[k]);
                    res_L.push_back(res[k]);
                }
                for (int k = 0, q = 0; k < nact; ++k) {
                    if (q < (int)done.size() && done[q] == k)
                        ++q;
                    else
                        keep.push_back(k);
                }
                gather_columns_impl(Y, ld, n, keep, cplx, Yalt, ld, s);
                std::swap(Y, Yalt);
                nl += (int)done.size();
            }
        }
        if (keep.empty()) {
            prev_theta.assign(theta.begin(), theta.begin() + nact);
            prev_res.assign(res.begin(), res.begin() + nact);
        } else {
            prev_theta.clear();
            prev_res.clear();
            for (int k : keep) {
                prev_theta.push_back(theta[k]);
                prev_res.push_back(res[k]);
            }
            nact = (int)keep.size();
        }
        if (single_phase) convert_block_impl(Y, d64, ld, X32.p, d32, ld, n, nact, s);
    }
    if (it > p.max_iter) it = p.max_iter;
    // ---- collect the accepted pairs (ascending theta: already sorted)
    if (nl > 0) {
        // the locked pairs and the accepted ones of the last iteration, ascending
        const int ew = cplx ? 2 : 1;
        gather_columns_impl(Y, ld, n, acc_idx, cplx, (double*)Lk.p + (size_t)nl * ew, ld, s);
        for (int k : acc_idx) {
            lam_L.push_back(theta[k]);
            res_L.push_back(res[k]);
        }
        std::vector<int> order(lam_L.size());
        for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return lam_L[x] < lam_L[y]; });
        fill_result(R, order, lam_L, res_L, Lk.p, n, ld, dtype_size(d64), it, converged,
                    fp64_its, n_mvm, a, b, s);
    } else {
        fill_result(R, acc_idx, theta, res, Y, n, ld, dtype_size(d64), it, converged, fp64_its,
                    n_mvm, a, b, s);
    }
    R->info.seconds_filter = t_filter;
    R->info.seconds_dense = t_dense;
    R->info.seconds_total = now() - t_start;
}

chebfd_result* new_result() { return new chebfd_result(); }

void set_iterations(chebfd_result* R, const std::vector<chebfd_iteration_info>& recs) {
    R->iterations = recs;
}

// Copy the accepted Ritz pairs (columns acc of the row-major block Y) into R.
void fill_result(chebfd_result* R, const std::vector<int>& acc, const std::vector<double>& theta,
                 const std::vector<double>& res, const void* Y, int64_t n, int64_t ld,
                 size_t es, int iterations, bool converged, int fp64_its, int64_t n_mvm,
                 double a, double b, cudaStream_t s) {
    const int nev = (int)acc.size();
    // the stream-ordered pool keeps the iteration's freed blocks; hand them
    // back before the result's own allocation
    {
        int dev = 0;
        cudaMemPool_t pool;
        CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess)
            cudaMemPoolTrimTo(pool, 0);
    }
    R->lambda.resize(nev);
    R->res.resize(nev);
    R->n = n;
    R->elem_size = es;
    if (nev > 0) {
        CHEBFD_CHECK_CUDA(cudaMalloc(&R->V, (size_t)n * nev * es));
        for (int q = 0; q < nev; ++q) {
            const int k = acc[q];
            R->lambda[q] = theta[k];
            R->res[q] = res[k];
            CHEBFD_CHECK_CUDA(cudaMemcpy2DAsync((char*)R->V + q * es, nev * es,
                                                (const char*)Y + k * es, ld * es, es, n,
                                                cudaMemcpyDeviceToDevice, s));
        }
        CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    chebfd_result_info& I = R->info;
    I.nev = nev;
    I.iterations = iterations;
    I.converged = converged ? 1 : 0;
    I.fp64_iterations = fp64_its;
    I.n_mvm = n_mvm;
    I.a = a;
    I.b = b;
    I.lambda = R->lambda.data();
    I.res = R->res.data();
    I.V = R->V;
}

void orthonormalize_impl(void* Yv, int64_t n, int ns, int64_t ld, chebfd_dtype dt,
                         uint64_t seed, int64_t* refill_counter, int* rank_out, cudaStream_t s);
void residuals_impl(const Matrix& M, const void* V, const double* theta_host, int64_t ld, int k,
                    chebfd_dtype dt, double* res_host, cudaStream_t s);

}  // namespace chebfd

using namespace chebfd;

extern "C" {

chebfd_status chebfd_orthonormalize(void* Y, int64_t n, int ns, int64_t ld, chebfd_dtype vdt,
                                    uint64_t refill_seed, int64_t* refill_counter, int* rank,
                                    void* stream) {
    return guarded([&] {
        orthonormalize_impl(Y, n, ns, ld, vdt, refill_seed, refill_counter, rank,
                            as_stream(stream));
    });
}

chebfd_status chebfd_rayleigh_ritz(const chebfd_matrix* H, void* Y, int64_t ld, int ns,
                                   chebfd_dtype vdt, double* theta, double* res, void* HV,
                                   void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        rayleigh_ritz_impl(H->m, Y, ld, ns, vdt, theta, res, HV, as_stream(stream));
    });
}

chebfd_status chebfd_harmonic_ritz(const chebfd_matrix* H, void* Y, int64_t ld, int ns,
                                   chebfd_dtype vdt, double tau, double* theta, double* res,
                                   void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        harmonic_ritz_impl(H->m, Y, ld, ns, vdt, tau, theta, res, as_stream(stream));
    });
}

chebfd_status chebfd_residuals(const chebfd_matrix* H, const void* V, const double* theta,
                               int64_t ld, int k, chebfd_dtype vdt, double* res, void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(H, CHEBFD_EINVAL, "null matrix");
        residuals_impl(H->m, V, theta, ld, k, vdt, res, as_stream(stream));
    });
}

chebfd_status chebfd_convert_block(const void* X, chebfd_dtype xdt, int64_t ldx, void* Y,
                                   chebfd_dtype ydt, int64_t ldy, int64_t n, int nb,
                                   void* stream) {
    return guarded(
        [&] { convert_block_impl(X, xdt, ldx, Y, ydt, ldy, n, nb, as_stream(stream)); });
}

chebfd_status chebfd_solve(const chebfd_matrix* H, const chebfd_params* p, void* stream,
                           chebfd_result** out) {
    chebfd_result* R = nullptr;
    chebfd_status st = guarded([&] {
        CHEBFD_REQUIRE(H && p && out, CHEBFD_EINVAL, "null argument");
        R = new chebfd_result();
        solve_impl(H->m, *p, as_stream(stream), R);
    });
    if (st != CHEBFD_OK) {
        if (R) {
            cudaFree(R->V);
            delete R;
        }
        return st;
    }
    *out = R;
    if (!R->info.converged) {
        set_error("ChebFD did not converge within max_iter iterations");
        return CHEBFD_ENOCONV;
    }
    return CHEBFD_OK;
}

chebfd_status chebfd_result_get(const chebfd_result* r, chebfd_result_info* out) {
    return guarded([&] {
        CHEBFD_REQUIRE(r && out, CHEBFD_EINVAL, "null argument");
        *out = r->info;
    });
}

chebfd_status chebfd_result_iterations(const chebfd_result* r, chebfd_iteration_info* out,
                                       int capacity, int* count) {
    return guarded([&] {
        CHEBFD_REQUIRE(r && count && capacity >= 0 && (out || capacity == 0), CHEBFD_EINVAL,
                       "bad argument");
        *count = (int)r->iterations.size();
        const int m = std::min(capacity, *count);
        for (int i = 0; i < m; ++i) out[i] = r->iterations[i];
    });
}

chebfd_status chebfd_result_copy_vectors(const chebfd_result* r, void* dst, int64_t ld,
                                         void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(r && (dst || r->info.nev == 0), CHEBFD_EINVAL, "null argument");
        const int nev = r->info.nev;
        CHEBFD_REQUIRE(ld >= nev, CHEBFD_EINVAL, "ld < nev");
        if (nev == 0) return;
        const size_t es = r->elem_size;
        cudaStream_t s = as_stream(stream);
        CHEBFD_CHECK_CUDA(cudaMemcpy2DAsync(dst, ld * es, r->V, nev * es, nev * es, r->n,
                                            cudaMemcpyDeviceToDevice, s));
        CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
    });
}

chebfd_status chebfd_result_destroy(chebfd_result* r) {
    return guarded([&] {
        if (!r) return;
        cudaFree(r->V);
        delete r;
    });
}

}  // extern "C"
