// Fused Chebyshev step (Fig. ChebFD, MODE_STEP) on the blocked-ELL copy of a
// complex matrix, complex64 vectors:  w = 2 (alpha H + beta) u - w ; y += c w.
//
// The rows of a block (the 4 orbitals of one lattice site) share their
// column blocks (the same 7 sites), so one group of G lanes computes all 4
// rows together: every gathered u row (nb complex64 = nb*8 bytes, one 16-byte
// chunk per lane) is loaded once and used by the 4 rows, which halves the
// L1 traffic of the gathers against the row-wise SELL kernel (28 instead of
// 52 row reads per site), and the dense 4x4 block values are read from
// shared memory with broadcast loads instead of shuffles.  beta enters as a shift
// beta/alpha of the diagonal block (slot 0), so the own row of u is not read
// a second time.  w and y of the 4 rows are prefetched to L2 when the block
// row starts and read after the products.
#include <algorithm>
#include <cstdlib>

#include "async_copy.cuh"
#include "filter_kernels.cuh"

namespace chebfd {

namespace {

constexpr int BELL_THREADS = 256;

struct BellView {
    const int32_t* bcol;  // [nbr][kBellLB]
    const float4* bval;   // [nbr][kBellLB][8]: 16 complex64 values, two per float4
    int64_t nbr;
};

__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }

// G lanes per block row; lane < wc owns one 16-byte chunk (two complex
// columns) of the 4 rows.  Block rows are visited in the same wave-front
// order as the SELL kernel (block b of wave w takes `tile` consecutive slot
// groups), with a block-uniform trip count so shuffles see full warps.
// The block values are staged in shared memory: each lane group copies the
// next block row's 7 blocks (896 bytes) with cp.async while it works on the
// current one (double buffer per group) and reads them with broadcast shared
// loads, so only the u gathers hold registers across memory latency (this
// took the kernel from 0.65 to 0.84 of the measured HBM bandwidth against
// keeping the values in registers).
// ENS: an ensemble of such matrices (block-diagonal); each block row reads
// its member's 2 alpha, g_n c_n and beta/alpha from the coefficient table.
template <int G, bool ENS>
__global__ void __launch_bounds__(BELL_THREADS, 2)
    bell_step_kernel(BellView H, StepArgs a, int wc, float shift) {
    constexpr int B = kBellB, LB = kBellLB, SLOTS = BELL_THREADS / G, NV = LB * 8;
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(G >= LB, "one lane per block column");
    extern __shared__ float4 sval[];  // [2][SLOTS][NV]
    const int lane = threadIdx.x % G, slot = threadIdx.x / G;
    const bool on = lane < wc;
    const float* __restrict__ u = reinterpret_cast<const float*>(a.gather);
    float* __restrict__ w = reinterpret_cast<float*>(a.w);
    float* __restrict__ y = reinterpret_cast<float*>(a.y);
    const int64_t ldg = 2 * a.ldg, ldw = 2 * a.ldw, ldy = 2 * a.ldy;
    const int64_t cofs = 4 * (int64_t)lane;
    float2 ta = dup((float)(2.0 * a.alpha)), cc = dup((float)a.c0);

    const int tile = a.tile > 0 ? a.tile : 1;
    const int64_t wave = (int64_t)gridDim.x * tile * SLOTS;
    const int iters = (int)((H.nbr + wave - 1) / wave) * tile;
    const int64_t wrap = wave - (int64_t)(tile - 1) * SLOTS;
    int64_t q = (int64_t)blockIdx.x * tile * SLOTS + slot;  // visit index; site = order.site(q)
    int tt = 0;

    auto stage = [&](int64_t row, int buf) {
        if (row < H.nbr) {
            float4* dst = sval + ((size_t)buf * SLOTS + slot) * NV;
            const float4* src = H.bval + row * NV;
#pragma unroll
            for (int j = lane; j < NV; j += G) cp_async16(dst + j, src + j);
        }
        cp_async_commit();
    };

    const int64_t s0 = q < H.nbr ? a.order.site(q) : H.nbr;
    int32_t bc_next = (s0 < H.nbr && lane < LB) ? __ldcs(H.bcol + s0 * LB + lane) : 0;
    stage(s0, 0);

    for (int it = 0; it < iters; ++it) {
        const int64_t q_next = tt + 1 == tile ? q + wrap : q + SLOTS;
        const bool active = q < H.nbr;
        const int64_t br = active ? a.order.site(q) : 0;
        const int64_t br_next = q_next < H.nbr ? a.order.site(q_next) : H.nbr;
        const int32_t bc_cur = bc_next;
        bc_next = (br_next < H.nbr && lane < LB) ? __ldcs(H.bcol + br_next * LB + lane) : 0;
        stage(br_next, (it + 1) & 1);
        if constexpr (ENS) {
            if (active) {
                const double* cf = a.coef + (int64_t)__ldg(a.row_inst + br * B) * a.coef_ld;
                ta = dup(2.0f * (float)__ldg(cf));  // == (float)(2 alpha): doubling is exact
                cc = dup((float)__ldg(cf + 2 + a.mom_step));
                shift = (float)__ldg(cf + a.coef_ld - 1);
            }
        }
        if (active && on) {
#pragma unroll
            for (int r = 0; r < B; ++r) {
                prefetch_l2(w + (br * B + r) * ldw + cofs);
                prefetch_l2(y + (br * B + r) * ldy + cofs);
            }
        }
        float2 P[B][2], Q[B][2];
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) P[r][c] = Q[r][c] = make_float2(0.f, 0.f);

        auto gather = [&](int k, float4* g) {
            const int32_t cj = __shfl_sync(FULL, bc_cur, k, G);
            const float* urow = u + (int64_t)cj * B * ldg + cofs;
#pragma unroll
            for (int o = 0; o < B; ++o)
                g[o] = (active && on) ? __ldg(reinterpret_cast<const float4*>(urow + o * ldg))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        cp_async_wait_prev();  // this block row's values (staged one iteration ago)
        __syncwarp();
        const float4* vb = sval + ((size_t)(it & 1) * SLOTS + slot) * NV;
#pragma unroll
        for (int k = 0; k < LB; ++k) {
            float4 g[B];
            gather(k, g);
#pragma unroll
            for (int o = 0; o < B; ++o) {
                const float2 ar = dup(g[o].x), ai = dup(g[o].y);
                const float2 cr = dup(g[o].z), ci = dup(g[o].w);
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    const int e = r * B + o;
                    const float4 q = vb[k * 8 + (e >> 1)];
                    float2 h = (e & 1) ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
                    if (k == 0 && r == o) h.x += shift;
                    P[r][0] = __ffma2_rn(h, ar, P[r][0]);
                    Q[r][0] = __ffma2_rn(h, ai, Q[r][0]);
                    P[r][1] = __ffma2_rn(h, cr, P[r][1]);
                    Q[r][1] = __ffma2_rn(h, ci, Q[r][1]);
                }
            }
        }
        __syncwarp();  // the next stage() may overwrite this buffer

        if (active && on) {
            float4 wo[B], yo[B];
#pragma unroll
            for (int r = 0; r < B; ++r) {
                wo[r] = __ldcs(reinterpret_cast<const float4*>(w + (br * B + r) * ldw + cofs));
                yo[r] = __ldcs(reinterpret_cast<const float4*>(y + (br * B + r) * ldy + cofs));
            }
#pragma unroll
            for (int r = 0; r < B; ++r) {
                const float2 h0 = make_float2(P[r][0].x - Q[r][0].y, P[r][0].y + Q[r][0].x);
                const float2 h1 = make_float2(P[r][1].x - Q[r][1].y, P[r][1].y + Q[r][1].x);
                const float2 w0 = __ffma2_rn(ta, h0, make_float2(-wo[r].x, -wo[r].y));
                const float2 w1 = __ffma2_rn(ta, h1, make_float2(-wo[r].z, -wo[r].w));
                const float2 y0 = __ffma2_rn(cc, w0, make_float2(yo[r].x, yo[r].y));
                const float2 y1 = __ffma2_rn(cc, w1, make_float2(yo[r].z, yo[r].w));
                __stcs(reinterpret_cast<float4*>(w + (br * B + r) * ldw + cofs),
                       make_float4(w0.x, w0.y, w1.x, w1.y));
                __stcs(reinterpret_cast<float4*>(y + (br * B + r) * ldy + cofs),
                       make_float4(y0.x, y0.y, y1.x, y1.y));
            }
        }
        q = q_next;
        tt = tt + 1 == tile ? 0 : tt + 1;
    }
    cp_async_wait_all();
}

template <int G, bool ENS>
void launch_g(const BellView& v, const StepArgs& a, int wc, float shift, int sms,
              cudaStream_t s) {
    constexpr int SLOTS = BELL_THREADS / G;
    const size_t smem = (size_t)2 * SLOTS * kBellLB * 8 * sizeof(float4);
    auto kern = bell_step_kernel<G, ENS>;
    ensure_dynamic_smem(reinterpret_cast<const void*>(kern), smem);
    const int grid = sms * std::min(8, cached_occupancy(reinterpret_cast<const void*>(kern),
                                                        BELL_THREADS, smem));
    kern<<<grid, BELL_THREADS, smem, s>>>(v, a, wc, shift);
}

}  // namespace

bool bell_step_applies(const Matrix& M, chebfd_dtype dt, StepMode mode, const StepArgs& a,
                       int wc) {
    return M.bell_enabled && M.bell_col != nullptr && dt == CHEBFD_C64 && mode == MODE_STEP &&
           a.moments == nullptr && (a.coef == nullptr || a.row_inst != nullptr) && wc >= 1 &&
           wc <= 32;
}

void launch_bell_step(const Matrix& M, const StepArgs& a, int wc, cudaStream_t s) {
    StepArgs b = a;
    static const int env_tile = [] {
        const char* e = getenv("CHEBFD_BELL_TILE");
        return e ? std::max(1, atoi(e)) : 1;
    }();
    b.tile = a.tile > 0 ? a.tile : env_tile;
    BellView v;
    v.bcol = M.bell_col;
    v.bval = reinterpret_cast<const float4*>(M.bell_val32);
    v.nbr = M.n / kBellB;
    const float shift = a.coef ? 0.f : (float)(a.beta / a.alpha);  // ensembles: per member
    const bool ens = a.coef != nullptr;
    if (wc > 16)
        ens ? launch_g<32, true>(v, b, wc, shift, M.num_sms, s)
            : launch_g<32, false>(v, b, wc, shift, M.num_sms, s);
    else if (wc > 8)
        ens ? launch_g<16, true>(v, b, wc, shift, M.num_sms, s)
            : launch_g<16, false>(v, b, wc, shift, M.num_sms, s);
    else
        ens ? launch_g<8, true>(v, b, wc, shift, M.num_sms, s)
            : launch_g<8, false>(v, b, wc, shift, M.num_sms, s);
}

}  // namespace chebfd
