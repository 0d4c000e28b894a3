// Parameter choice for ChebFD (Sec. 3.1 steps 1-3) from a KPM estimate of the
// DOS: the paper's rules (heuristic) or the trained MLP (learned parameters).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace chebfd {

void kpm_impl(const Matrix& M, double alpha, double beta, int Mm, int R, uint64_t seed,
              double* mu, cudaStream_t s);
void scale_bounds_impl(const Matrix& M, int steps, uint64_t seed, double* a_out, double* b_out,
                       cudaStream_t s);
void solve_impl(const Matrix& M, const chebfd_params& p0, cudaStream_t s, chebfd_result* R);

namespace {

constexpr int kCountMoments = 1024;  // KPM resolution for the window counts
constexpr int kProbes = 8;

// N_0 of the Lanczos kernel (mu = 2) at interval centre c / S_w = 0, 0.1, ..., 0.9
// (Tab. lanczoskernel); linear interpolation in between, the last value beyond.
double lanczos_N0(double rel_centre) {
    static const double tab[10] = {6.23, 6.20, 6.10, 5.94, 5.71, 5.40, 4.99, 4.46, 3.75, 2.73};
    const double x = std::min(std::fabs(rel_centre), 0.9) * 10.0;
    const int i = std::min((int)x, 8);
    const double f = x - i;
    return tab[i] * (1.0 - f) + tab[i + 1] * f;
}

// KPM count of eigenvalues in [lo, hi] (Eq. DOS:target): N sum_n g_n mu_n c_n,
// Jackson factors for the moment count (Tab. Kernel with N_p = M + 1).
double kpm_count(const std::vector<double>& mu, int64_t N, double a, double b, double lo,
                 double hi) {
    const int Mm = (int)mu.size();
    std::vector<double> c(Mm);
    lo = std::max(lo, a);
    hi = std::min(hi, b);
    if (!(hi > lo)) return 0.0;
    const chebfd_status st =
        chebfd_window_coeffs(a, b, lo, hi, Mm - 1, CHEBFD_KERNEL_NONE, 0.0, c.data());
    CHEBFD_REQUIRE(st == CHEBFD_OK, st, "window coefficients failed");
    const double pi = 3.14159265358979323846;
    const int Nk = Mm + 1;
    double s = 0.0;
    for (int n = 0; n < Mm; ++n) {
        const double q = pi / Nk;
        const double g = ((Nk - n) * std::cos(q * n) + std::sin(q * n) / std::tan(q)) / Nk;
        s += g * mu[n] * c[n];
    }
    return (double)N * s;
}

struct Analysis {
    double a, b, alpha, beta, n_target;
    std::vector<double> mu;
};

Analysis analyse(const Matrix& M, double a, double b, double lo, double hi, uint64_t seed,
                 cudaStream_t s) {
    Analysis A;
    if (!(b > a)) scale_bounds_impl(M, 30, seed, &a, &b, s);
    A.a = a;
    A.b = b;
    A.alpha = 2.0 / (b - a);
    A.beta = (a + b) / (a - b);
    A.mu.resize(kCountMoments);
    kpm_impl(M, A.alpha, A.beta, kCountMoments, kProbes, seed, A.mu.data(), s);
    A.n_target = std::max(0.0, kpm_count(A.mu, M.n, a, b, lo, hi));
    return A;
}

// Never fewer search vectors than target vectors (Sec. 3.1 step 2 needs
// N_S > N_T): at least the KPM estimate N_T plus 8 for its stochastic error,
// rounded up to a multiple of 8, and at least 16.
int ns_floor(const Analysis& A) {
    const int f = (int)std::ceil((std::max(A.n_target, 0.0) + 8.0) / 8.0) * 8;
    return std::max(16, std::min(f, 1024));
}

void heuristic(const Matrix& M, const Analysis& A, double lo, double hi, int* ns, int* Np,
               int* kernel) {
    // Sec. 3.1 step 2 / Sec. 2.4: N_S = 4 N_T (optimum for the linear DOS of
    // the insulator and graphene), a multiple of 8, at least 16
    int n_s = (int)std::ceil(4.0 * std::max(A.n_target, 1.0) / 8.0) * 8;
    n_s = std::max(ns_floor(A), std::min(n_s, 1024));
    // Step 3, Eq. DOS:search: the margin delta' at which the KPM count reaches N_S
    double d_lo = 0.0, d_hi = A.b - A.a;
    for (int it = 0; it < 60; ++it) {
        const double d = 0.5 * (d_lo + d_hi);
        if (kpm_count(A.mu, M.n, A.a, A.b, lo - d, hi + d) < n_s)
            d_lo = d;
        else
            d_hi = d;
    }
    const double dprime = std::max(0.5 * (d_lo + d_hi), 1e-12);
    // N_p = N_0 S_w / delta' (Eq. etafit), N_0 of Tab. lanczoskernel at the window centre
    const double S_w = 0.5 * (A.b - A.a);
    const double centre = 0.5 * (lo + hi) - 0.5 * (A.a + A.b);
    const double n_p = lanczos_N0(centre / S_w) * S_w / dprime;
    *Np = (int)std::max(8.0, std::min(20000.0, std::round(n_p)));
    *ns = n_s;
    *kernel = CHEBFD_KERNEL_LANCZOS;
}

}  // namespace

// Adaptive degree (the adaptive choice of N_p suggested in Sec. 6, with the
// rule of Sec. 2.4): mu are the normalised moments the first filter returned
// for the n_s random search vectors (a stochastic-trace KPM estimate, at
// most 1024 used); N_T from the window count, delta' where the count of the
// search interval reaches n_s, N_p = N_0 S_w / delta' within [Np0/4, 4 Np0].
int adaptive_degree(const std::vector<double>& mu_in, int64_t N, double a, double b, double lo,
                    double hi, int ns, int Np0, double* n_target, double* dprime_out) {
    const std::vector<double> mu(mu_in.begin(),
                                 mu_in.begin() + std::min<size_t>(mu_in.size(), kCountMoments));
    if (n_target) *n_target = std::max(0.0, kpm_count(mu, N, a, b, lo, hi));
    double d_lo = 0.0, d_hi = b - a;
    for (int it = 0; it < 60; ++it) {
        const double d = 0.5 * (d_lo + d_hi);
        if (kpm_count(mu, N, a, b, lo - d, hi + d) < ns)
            d_lo = d;
        else
            d_hi = d;
    }
    const double dprime = std::max(0.5 * (d_lo + d_hi), 1e-12);
    if (dprime_out) *dprime_out = dprime;
    const double S_w = 0.5 * (b - a);
    const double centre = 0.5 * (lo + hi) - 0.5 * (a + b);
    const double n_p = std::round(lanczos_N0(centre / S_w) * S_w / dprime);
    return (int)std::min<double>(std::max<double>(n_p, std::max(2, Np0 / 4)), 4.0 * Np0);
}

void features_of(const Matrix& M, const Analysis& A, double lo, double hi, int m_feat,
                 double* f) {
    for (int n = 0; n < m_feat; ++n) f[n] = n < (int)A.mu.size() ? A.mu[n] : 0.0;
    f[m_feat] = A.alpha * 0.5 * (lo + hi) + A.beta;                 // window centre in [-1, 1]
    f[m_feat + 1] = std::log10(std::max(A.alpha * 0.5 * (hi - lo), 1e-12));  // half width
    f[m_feat + 2] = std::log10(std::max(A.n_target, 1.0));         // wanted count
}

}  // namespace chebfd

using namespace chebfd;

extern "C" {

chebfd_status chebfd_mlp_forward(chebfd_mlp* N, const float* X, int B, float* Z, void* stream);

chebfd_status chebfd_param_features(const chebfd_matrix* H, double a, double b, double lam_lo,
                                    double lam_hi, int m_feat, uint64_t seed, double* features,
                                    double* n_target, void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(H && features && m_feat >= 2 && m_feat <= kCountMoments, CHEBFD_EINVAL,
                       "bad feature arguments");
        CHEBFD_REQUIRE(lam_hi > lam_lo, CHEBFD_EINVAL, "need lam_hi > lam_lo");
        const Analysis A = analyse(H->m, a, b, lam_lo, lam_hi, seed, as_stream(stream));
        features_of(H->m, A, lam_lo, lam_hi, m_feat, features);
        if (n_target) *n_target = A.n_target;
    });
}

chebfd_status chebfd_choose_params(const chebfd_matrix* H, double a, double b, double lam_lo,
                                   double lam_hi, chebfd_mlp* mlp, int m_feat, uint64_t seed,
                                   int* ns, int* Np, int* kernel, double* n_target,
                                   void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(H && ns && Np && kernel, CHEBFD_EINVAL, "null argument");
        CHEBFD_REQUIRE(lam_hi > lam_lo, CHEBFD_EINVAL, "need lam_hi > lam_lo");
        cudaStream_t s = as_stream(stream);
        const Analysis A = analyse(H->m, a, b, lam_lo, lam_hi, seed, s);
        if (n_target) *n_target = A.n_target;
        if (!mlp) {
            heuristic(H->m, A, lam_lo, lam_hi, ns, Np, kernel);
            return;
        }
        CHEBFD_REQUIRE(m_feat >= 2 && m_feat <= kCountMoments, CHEBFD_EINVAL, "bad m_feat");
        std::vector<double> f(m_feat + 3);
        features_of(H->m, A, lam_lo, lam_hi, m_feat, f.data());
        std::vector<float> ff(f.begin(), f.end());
        float *dx = nullptr, *dz = nullptr;
        CHEBFD_CHECK_CUDA(cudaMalloc(&dx, ff.size() * sizeof(float)));
        CHEBFD_CHECK_CUDA(cudaMalloc(&dz, 3 * sizeof(float)));
        float z[3] = {0.f, 0.f, 0.f};
        chebfd_status st = CHEBFD_OK;
        if (cudaMemcpyAsync(dx, ff.data(), ff.size() * sizeof(float), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            st = CHEBFD_ECUDA;
        if (st == CHEBFD_OK) st = chebfd_mlp_forward(mlp, dx, 1, dz, stream);
        if (st == CHEBFD_OK &&
            (cudaMemcpyAsync(z, dz, sizeof(z), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
             cudaStreamSynchronize(s) != cudaSuccess))
            st = CHEBFD_ECUDA;
        cudaFree(dx);
        cudaFree(dz);
        CHEBFD_REQUIRE(st == CHEBFD_OK, st, "MLP inference failed");
        // outputs are scale-free: log(N_p / N_p of the rule), log(n_s / N_T),
        // kernel logit (> 0: Lanczos, else Jackson); each is kept inside the
        // range the network was trained on (N_p ratio [1/2, 2], n_s/N_T [2, 6],
        // the paper's 2 <= N_S/N_T recommendation at the low end)
        int ns_rule = 0, np_rule = 0, k_rule = 0;
        heuristic(H->m, A, lam_lo, lam_hi, &ns_rule, &np_rule, &k_rule);
        const double rp = std::exp(std::max(std::log(0.5), std::min(std::log(2.0), (double)z[0])));
        const double rs = std::exp(std::max(std::log(2.0), std::min(std::log(6.0), (double)z[1])));
        *Np = (int)std::max(8.0, std::min(20000.0, std::round(rp * np_rule)));
        const int n_s = (int)std::ceil(rs * std::max(A.n_target, 1.0) / 8.0) * 8;
        *ns = std::max(ns_floor(A), std::min(n_s, 1024));
        *kernel = z[2] > 0.f ? CHEBFD_KERNEL_LANCZOS : CHEBFD_KERNEL_JACKSON;
    });
}

}  // extern "C"
