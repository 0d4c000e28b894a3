// Matrix-free Chebyshev steps (MODE_STEP) for the insulator lattices, in
// complex64 and in double-float arithmetic: w = 2 (alpha H + beta) u - w ;
// y += c w with H's entries rebuilt in registers from the lattice
// description instead of read from memory (the paper's on-the-fly matrices,
// Sec. 1).
//
// Same mapping as the blocked step (step_bell.cu): one group of G lanes per
// site computes its 4 orbital rows, each lane one 16-byte chunk (two complex
// columns), gathering each neighbour site's 4 rows once.  The entries follow
// the generator: onsite (m + V_s) Gamma1 (TOPI) or V_s + m Gamma1 (TOPI_SLAB)
// with V_s regenerated from the SplitMix64 disorder stream, and for each
// axis j the hopping block T_j = -(t/2)(Gamma1 - i Gamma_{j+1}) at the site
// below and T_j^dagger at the site above: row o couples to orbital o with
// -(t/2) Gamma1[o][o] and to its Gamma_{j+1} partner p with a purely real or
// purely imaginary value.  Only the vectors move: 5 n_b S_v bytes per row.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "async_copy.cuh"
#include "df.cuh"
#include "filter_kernels.cuh"

namespace chebfd {

namespace {

constexpr int ST_THREADS = 256;

struct StencilView {
    int64_t Lx, Ly, Lz, nsite;
    float h;        // t / 2
    double hd;      // t / 2 in FP64 (double-float step)
    double m, W;
    uint64_t seed;
    int slab;       // open in z
};

__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

// acc += a u (real a) and acc += i b u (imaginary b) on a 16-byte chunk of two
// complex entries held as two float2 (re, im).
__device__ __forceinline__ void mac_re(float2* acc, float a, const float4& u) {
    acc[0] = __ffma2_rn(dup2(a), make_float2(u.x, u.y), acc[0]);
    acc[1] = __ffma2_rn(dup2(a), make_float2(u.z, u.w), acc[1]);
}
__device__ __forceinline__ void mac_im(float2* acc, float b, const float4& u) {
    const float2 bb = make_float2(-b, b);
    acc[0] = __ffma2_rn(bb, make_float2(u.y, u.x), acc[0]);
    acc[1] = __ffma2_rn(bb, make_float2(u.w, u.z), acc[1]);
}

// Add the hopping block of axis j (0, 1, 2) from a neighbour site whose 4
// rows are g: q = +1 for the site below (T_j), -1 for the site above (T_j^dagger).
template <int J>
__device__ __forceinline__ void hop(float2 (*acc)[2], const float4* g, float h, float q) {
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const bool upper = o < 2;
        mac_re(acc[o], upper ? -h : h, g[o]);  // -h Gamma1[o][o]
        // partner p and Gamma_{j+1}[o][p] = gr + i gi; entry q i h (gr + i gi)
        if (J == 0) {        // sx (x) sx: real 1
            mac_im(acc[o], q * h, g[o ^ 3]);
        } else if (J == 1) { // sx (x) sy: -i for o = 0, 2; +i for o = 1, 3
            const float gi = (o == 0 || o == 2) ? -1.f : 1.f;
            mac_re(acc[o], -q * h * gi, g[o ^ 3]);
        } else {             // sx (x) sz: +1 for o = 0, 2; -1 for o = 1, 3
            const float gr = (o == 0 || o == 2) ? 1.f : -1.f;
            mac_im(acc[o], q * h * gr, g[o ^ 2]);
        }
    }
}

// (H + shift) u on the 4 rows of site s = (x, y, z) for one 16-byte chunk of
// columns, accumulated in acc[row][2]: the onsite block first, then the
// neighbours -x, +x, -y, +y, -z, +z (the slab has no z neighbour beyond its
// faces).  gather(k, g) loads the 4 rows of neighbour k (0: the site itself,
// 1..6 in that order) into g.  The same order everywhere, so every caller
// rounds alike.
template <class Gather>
__device__ __forceinline__ void stencil_site_acc(const StencilView& L, int64_t s, int64_t z,
                                                 float shift, Gather&& gather,
                                                 float2 (*acc)[2]) {
    constexpr int B = 4;
#pragma unroll
    for (int r = 0; r < B; ++r) acc[r][0] = acc[r][1] = make_float2(0.f, 0.f);
    float4 g[B];
    gather(0, g);
    // the generator's roundings: V = W (u - 1/2), then m + V or V +- m
    const double V = __dmul_rn(L.W, splitmix_uniform(L.seed, STREAM_DISORDER, (uint64_t)s) - 0.5);
    float on_up, on_lo;
    if (L.slab) {
        on_up = __double2float_rn(__dadd_rn(V, L.m));
        on_lo = __double2float_rn(__dadd_rn(V, -L.m));
    } else {
        on_up = __double2float_rn(__dadd_rn(L.m, V));
        on_lo = -on_up;
    }
#pragma unroll
    for (int o = 0; o < B; ++o) mac_re(acc[o], (o < 2 ? on_up : on_lo) + shift, g[o]);
    gather(1, g);
    hop<0>(acc, g, L.h, 1.f);
    gather(2, g);
    hop<0>(acc, g, L.h, -1.f);
    gather(3, g);
    hop<1>(acc, g, L.h, 1.f);
    gather(4, g);
    hop<1>(acc, g, L.h, -1.f);
    if (!L.slab || z > 0) {
        gather(5, g);
        hop<2>(acc, g, L.h, 1.f);
    }
    if (!L.slab || z + 1 < L.Lz) {
        gather(6, g);
        hop<2>(acc, g, L.h, -1.f);
    }
}

template <int G>
__global__ void __launch_bounds__(ST_THREADS, 3)
    stencil_step_kernel(StencilView L, StepArgs a, int wc, float shift) {
    constexpr int B = 4, SLOTS = ST_THREADS / G;
    const int lane = threadIdx.x % G, slot = threadIdx.x / G;
    const bool on = lane < wc;
    const float* __restrict__ u = reinterpret_cast<const float*>(a.gather);
    float* __restrict__ w = reinterpret_cast<float*>(a.w);
    float* __restrict__ y = reinterpret_cast<float*>(a.y);
    const int64_t ldg = 2 * a.ldg, ldw = 2 * a.ldw, ldy = 2 * a.ldy;  // floats per row
    const int64_t cofs = 4 * (int64_t)lane;
    const float2 ta = dup2((float)(2.0 * a.alpha)), cc = dup2((float)a.c0);

    const int tile = a.tile > 0 ? a.tile : 1;
    const int64_t wave = (int64_t)gridDim.x * tile * SLOTS;
    const int iters = (int)((L.nsite + wave - 1) / wave) * tile;
    const int64_t wrap = wave - (int64_t)(tile - 1) * SLOTS;
    int64_t q = (int64_t)blockIdx.x * tile * SLOTS + slot;  // visit index; site = order.site(q)
    int tt = 0;

    for (int it = 0; it < iters; ++it) {
        const int64_t q_next = tt + 1 == tile ? q + wrap : q + SLOTS;
        if (q < L.nsite && on) {
            const int64_t s = a.order.site(q);
#pragma unroll
            for (int r = 0; r < B; ++r) {
                prefetch_l2(w + (s * B + r) * ldw + cofs);
                prefetch_l2(y + (s * B + r) * ldy + cofs);
            }
            const int si = (int)s, Lx = (int)L.Lx, Ly = (int)L.Ly;  // sites < 2^29
            const int64_t x = si % Lx, yy = (si / Lx) % Ly, z = si / (Lx * Ly);
            auto site = [&](int64_t cx, int64_t cy, int64_t cz) {
                return cx + L.Lx * (cy + L.Ly * cz);
            };
            // neighbour k of the site: 0 itself, 1..6 = -x, +x, -y, +y, -z, +z (periodic)
            auto gather = [&](int k, float4* g) {
                int64_t cx = x, cy = yy, cz = z;
                if (k == 1) cx = (x + L.Lx - 1) % L.Lx;
                if (k == 2) cx = (x + 1) % L.Lx;
                if (k == 3) cy = (yy + L.Ly - 1) % L.Ly;
                if (k == 4) cy = (yy + 1) % L.Ly;
                if (k == 5) cz = (z + L.Lz - 1) % L.Lz;
                if (k == 6) cz = (z + 1) % L.Lz;
                const float* base = u + site(cx, cy, cz) * B * ldg + cofs;
#pragma unroll
                for (int o = 0; o < B; ++o)
                    g[o] = __ldg(reinterpret_cast<const float4*>(base + o * ldg));
            };
            float2 acc[B][2];
            stencil_site_acc(L, s, z, shift, gather, acc);
#pragma unroll
            for (int r = 0; r < B; ++r) {
                const int64_t row = s * B + r;
                const float4 wo = __ldcs(reinterpret_cast<const float4*>(w + row * ldw + cofs));
                const float4 yo = __ldcs(reinterpret_cast<const float4*>(y + row * ldy + cofs));
                const float2 w0 = __ffma2_rn(ta, acc[r][0], make_float2(-wo.x, -wo.y));
                const float2 w1 = __ffma2_rn(ta, acc[r][1], make_float2(-wo.z, -wo.w));
                const float2 y0 = __ffma2_rn(cc, w0, make_float2(yo.x, yo.y));
                const float2 y1 = __ffma2_rn(cc, w1, make_float2(yo.z, yo.w));
                __stcs(reinterpret_cast<float4*>(w + row * ldw + cofs),
                       make_float4(w0.x, w0.y, w1.x, w1.y));
                __stcs(reinterpret_cast<float4*>(y + row * ldy + cofs),
                       make_float4(y0.x, y0.y, y1.x, y1.y));
            }
        }
        q = q_next;
        tt = tt + 1 == tile ? 0 : tt + 1;
    }
}

// ---- two Chebyshev steps per pass (temporal blocking of the matrix-free
// step; the paper's matrices constructed on the fly, Sec. 1) --------------
//
// u1 = 2 (alpha H + beta) u0 - um and u2 = 2 (alpha H + beta) u1 - u0 with
// y += c1 u1 + c2 u2, for a 16-column complex64 panel.  A CTA owns an 8 x 8
// tile of the x-y plane and Z consecutive z-planes.  Plane by plane it
// computes u1 on the tile and a one-site halo into a ring of three planes in
// shared memory (step 1, gathering u0 from global memory), then u2 on the
// tile one plane behind (step 2, gathering u1 from the ring).  u1 of the
// tile's own sites and u2 go to two other buffers (neighbouring CTAs still
// read u0 and um), y is read and written once.  Per pair of steps the
// vectors move 6 times instead of 10; the halo costs step-1 arithmetic
// (100 / 64 sites, (Z + 2) / Z planes).  Same per-site arithmetic as the
// single step, so a pair equals two single steps bit for bit.
constexpr int S2_TX = 8, S2_TY = 8;
constexpr int S2_HX = S2_TX + 2, S2_HY = S2_TY + 2, S2_HS = S2_HX * S2_HY;  // haloed sites
constexpr int S2_WC = 8;                          // 16-byte chunks per row: n_b = 16
constexpr int S2_THREADS = 256, S2_SLOTS = S2_THREADS / S2_WC;
constexpr size_t S2_RING_BYTES = (size_t)3 * S2_HS * 4 * S2_WC * 16;   // 153600

struct S2Args {
    const float* u0;   // T_n X   (gathered)
    const float* um;   // T_{n-1} X
    float* u1;         // out: T_{n+1} X
    float* u2;         // out: T_{n+2} X
    float* y;          // accumulated sum (in/out)
    int64_t ldw, ldy;  // floats per row of the work panels / of y
    float ta, shift, c1, c2;
    int Z;             // planes per CTA
};

__global__ void __launch_bounds__(S2_THREADS, 1) stencil2_kernel(StencilView L, S2Args a) {
    constexpr int B = 4;
    extern __shared__ float4 ring[];  // [3][S2_HS][B][S2_WC]
    const int lane = threadIdx.x % S2_WC, slot = threadIdx.x / S2_WC;
    const int tiles_x = (int)(L.Lx / S2_TX), tiles_y = (int)(L.Ly / S2_TY);
    const int tile = blockIdx.x % (tiles_x * tiles_y), seg = blockIdx.x / (tiles_x * tiles_y);
    const int x0 = (tile % tiles_x) * S2_TX, y0 = (tile / tiles_x) * S2_TY, z0 = seg * a.Z;
    const int Lx = (int)L.Lx, Ly = (int)L.Ly, Lz = (int)L.Lz;
    auto mod = [](int v, int n) { v %= n; return v < 0 ? v + n : v; };
    auto site = [&](int x, int y, int z) { return (int64_t)x + L.Lx * ((int64_t)y + L.Ly * z); };
    auto plane = [&](int zz) { return ring + (size_t)mod(zz - z0 + 1, 3) * S2_HS * B * S2_WC; };
    const float2 ta = dup2(a.ta), c1 = dup2(a.c1), c2 = dup2(a.c2);
    const int cofs = 4 * lane;
    for (int zz = z0 - 1; zz <= z0 + a.Z; ++zz) {
        // ---- step 1: u1 on the haloed plane zz (absent beyond a slab's faces)
        const bool exists = !L.slab || (zz >= 0 && zz < Lz);
        const int zw = mod(zz, Lz);
        float4* pz = plane(zz);
        for (int hs = slot; hs < S2_HS; hs += S2_SLOTS) {
            const int hx = hs % S2_HX, hy = hs / S2_HX;
            float4 out[B];
#pragma unroll
            for (int r = 0; r < B; ++r) out[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (exists) {
                const int gx = mod(x0 - 1 + hx, Lx), gy = mod(y0 - 1 + hy, Ly);
                const int64_t s = site(gx, gy, zw);
                auto gather = [&](int k, float4* g) {
                    int cx = gx, cy = gy, cz = zw;
                    if (k == 1) cx = mod(gx - 1, Lx);
                    if (k == 2) cx = mod(gx + 1, Lx);
                    if (k == 3) cy = mod(gy - 1, Ly);
                    if (k == 4) cy = mod(gy + 1, Ly);
                    if (k == 5) cz = mod(zw - 1, Lz);
                    if (k == 6) cz = mod(zw + 1, Lz);
                    const float* base = a.u0 + site(cx, cy, cz) * B * a.ldw + cofs;
#pragma unroll
                    for (int o = 0; o < B; ++o)
                        g[o] = __ldg(reinterpret_cast<const float4*>(base + o * a.ldw));
                };
                float2 acc[B][2];
                stencil_site_acc(L, s, zw, a.shift, gather, acc);
                const bool own = hx >= 1 && hx <= S2_TX && hy >= 1 && hy <= S2_TY && zz >= z0 &&
                                 zz < z0 + a.Z;
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    const int64_t row = s * B + r;
                    const float4 wo =
                        __ldg(reinterpret_cast<const float4*>(a.um + row * a.ldw + cofs));
                    const float2 w0 = __ffma2_rn(ta, acc[r][0], make_float2(-wo.x, -wo.y));
                    const float2 w1 = __ffma2_rn(ta, acc[r][1], make_float2(-wo.z, -wo.w));
                    out[r] = make_float4(w0.x, w0.y, w1.x, w1.y);
                    if (own) __stcs(reinterpret_cast<float4*>(a.u1 + row * a.ldw + cofs), out[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < B; ++r) pz[(hs * B + r) * S2_WC + lane] = out[r];
        }
        __syncthreads();
        // ---- step 2: u2 on the tile of plane zz - 1
        const int zt = zz - 1;
        if (zt >= z0 && zt < z0 + a.Z) {
            const int ztw = mod(zt, Lz);
            const float4* pm = plane(zt - 1);
            const float4* p0 = plane(zt);
            const float4* pp = plane(zt + 1);
            for (int ts = slot; ts < S2_TX * S2_TY; ts += S2_SLOTS) {
                const int tx = ts % S2_TX, ty = ts / S2_TX, hx = tx + 1, hy = ty + 1;
                const int64_t s = site(x0 + tx, y0 + ty, ztw);
                auto gather = [&](int k, float4* g) {
                    const float4* pl = k == 5 ? pm : (k == 6 ? pp : p0);
                    int cx = hx, cy = hy;
                    if (k == 1) cx = hx - 1;
                    if (k == 2) cx = hx + 1;
                    if (k == 3) cy = hy - 1;
                    if (k == 4) cy = hy + 1;
                    const float4* base = pl + (size_t)((cy * S2_HX + cx) * B) * S2_WC + lane;
#pragma unroll
                    for (int o = 0; o < B; ++o) g[o] = base[o * S2_WC];
                };
                float2 acc[B][2];
                stencil_site_acc(L, s, ztw, a.shift, gather, acc);
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    const int64_t row = s * B + r;
                    const float4 u1v = p0[((hy * S2_HX + hx) * B + r) * S2_WC + lane];
                    const float4 u0v =
                        __ldg(reinterpret_cast<const float4*>(a.u0 + row * a.ldw + cofs));
                    const float4 yo =
                        __ldcs(reinterpret_cast<const float4*>(a.y + row * a.ldy + cofs));
                    // the two single steps' updates of y, in their order
                    const float2 y0a = __ffma2_rn(c1, make_float2(u1v.x, u1v.y), make_float2(yo.x, yo.y));
                    const float2 y1a = __ffma2_rn(c1, make_float2(u1v.z, u1v.w), make_float2(yo.z, yo.w));
                    const float2 w0 = __ffma2_rn(ta, acc[r][0], make_float2(-u0v.x, -u0v.y));
                    const float2 w1 = __ffma2_rn(ta, acc[r][1], make_float2(-u0v.z, -u0v.w));
                    const float2 y0 = __ffma2_rn(c2, w0, y0a);
                    const float2 y1 = __ffma2_rn(c2, w1, y1a);
                    __stcs(reinterpret_cast<float4*>(a.u2 + row * a.ldw + cofs),
                           make_float4(w0.x, w0.y, w1.x, w1.y));
                    __stcs(reinterpret_cast<float4*>(a.y + row * a.ldy + cofs),
                           make_float4(y0.x, y0.y, y1.x, y1.y));
                }
            }
        }
        __syncthreads();
    }
}

template <int G>
void launch_g(const StencilView& v, const StepArgs& a, int wc, float shift, int sms,
              cudaStream_t s) {
    auto kern = stencil_step_kernel<G>;
    const int grid =
        sms * std::min(8, cached_occupancy(reinterpret_cast<const void*>(kern), ST_THREADS, 0));
    kern<<<grid, ST_THREADS, 0, s>>>(v, a, wc, shift);
}

// ---- double-float variant (the FP64-class sweep of MIXED_DF) -------------
//
// One lane owns one double-float complex entry (16 bytes: hi (re, im), lo
// (re, im)) of the 4 rows; every entry of H is real or imaginary, so each is
// one scalar-by-pair double-float multiply-add (13 per row) against two in
// the SELL double-float kernel.  The onsite value carries the shift
// beta/alpha (summed in FP64, then split).

__device__ __forceinline__ DFPair df_pair(const float4& c) {
    DFPair p;
    p.hi = make_float2(c.x, c.y);
    p.lo = make_float2(c.z, c.w);
    return p;
}
// i u for a complex pair u = (re, im): (-im, re)
__device__ __forceinline__ DFPair df_times_i(const DFPair& u) {
    DFPair r;
    r.hi = make_float2(-u.hi.y, u.hi.x);
    r.lo = make_float2(-u.lo.y, u.lo.x);
    return r;
}

template <int J>
__device__ __forceinline__ void hop_df(DFPair* acc, const float4* g, float h1, float h2, float q) {
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const float sd = o < 2 ? -1.f : 1.f;
        df_mac(acc[o], sd * h1, sd * h2, df_pair(g[o]));
        if (J == 0) {
            df_mac(acc[o], q * h1, q * h2, df_times_i(df_pair(g[o ^ 3])));
        } else if (J == 1) {
            const float gi = (o == 0 || o == 2) ? q : -q;
            df_mac(acc[o], gi * h1, gi * h2, df_pair(g[o ^ 3]));
        } else {
            const float gr = (o == 0 || o == 2) ? q : -q;
            df_mac(acc[o], gr * h1, gr * h2, df_times_i(df_pair(g[o ^ 2])));
        }
    }
}

// Unit-coefficient hopping sums of one neighbour (axis J, q = +1 below, -1
// above) for the exact-hopping path: with every hopping value +-h or +-i h,
// row o of H u gathers h S_o, where S_o sums the terms -+ g[o] of every
// neighbour and the partner terms (x: q i g[o^3], y: +-g[o^3], z: +-i
// g[o^2]).  The coefficients are +-1 and +-i, so each term is an error-free
// add (df_add_scaled); an imaginary term enters with its components
// swapped, i (a + i b) = (-b, a).
template <int J>
__device__ __forceinline__ void hop_sum_df(DFPair* S, const float4* g, float q, bool first) {
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const float sd = o < 2 ? -1.f : 1.f;
        const float sp = (o == 0 || o == 2) ? q : -q;
        const DFPair go = df_pair(g[o]);
        if (first) {
            S[o].hi = __fmul2_rn(make_float2(sd, sd), go.hi);
            S[o].lo = __fmul2_rn(make_float2(sd, sd), go.lo);
        } else {
            df_add_scaled(S[o], make_float2(sd, sd), go);
        }
        if (J == 0 || J == 2) {
            const float4 c = g[J == 0 ? o ^ 3 : o ^ 2];
            const float sg = J == 0 ? q : sp;
            const DFPair ic = {make_float2(c.y, c.x), make_float2(c.w, c.z)};
            df_add_scaled(S[o], make_float2(-sg, sg), ic);
        } else {
            df_add_scaled(S[o], make_float2(sp, sp), df_pair(g[o ^ 3]));
        }
    }
}

// a.ldg / a.ldw / a.ldy in 16-byte chunks (one double-float complex entry).
// EXACT: the hopping t/2 is a power of two (no low word, every product by it
// exact), so the hops are summed with unit coefficients and scaled once.
template <int G, int MINB, bool EXACT>
__global__ void __launch_bounds__(ST_THREADS, MINB)
    stencil_df_kernel(StencilView L, StepArgs a, int wc, double shift) {
    constexpr int B = 4, SLOTS = ST_THREADS / G;
    const int lane = threadIdx.x % G, slot = threadIdx.x / G;
    const bool on = lane < wc;
    const float4* __restrict__ u = reinterpret_cast<const float4*>(a.gather);
    float4* __restrict__ w = reinterpret_cast<float4*>(a.w);
    float4* __restrict__ y = reinterpret_cast<float4*>(a.y);
    const int64_t ldg = a.ldg, ldw = a.ldw, ldy = a.ldy;
    float ta1, ta2, c1, c2, h1, h2;
    df_split(2.0 * a.alpha, ta1, ta2);
    df_split(a.c0, c1, c2);
    df_split(L.hd, h1, h2);

    const int tile = a.tile > 0 ? a.tile : 1;
    const int64_t wave = (int64_t)gridDim.x * tile * SLOTS;
    const int iters = (int)((L.nsite + wave - 1) / wave) * tile;
    const int64_t wrap = wave - (int64_t)(tile - 1) * SLOTS;
    int64_t q = (int64_t)blockIdx.x * tile * SLOTS + slot;
    int tt = 0;

    for (int it = 0; it < iters; ++it) {
        const int64_t q_next = tt + 1 == tile ? q + wrap : q + SLOTS;
        if (q < L.nsite && on) {
            const int64_t s = a.order.site(q);
#pragma unroll
            for (int r = 0; r < B; ++r) {
                prefetch_l2(w + (s * B + r) * ldw + lane);
                prefetch_l2(y + (s * B + r) * ldy + lane);
            }
            const int si = (int)s, Lx = (int)L.Lx, Ly = (int)L.Ly;
            const int64_t x = si % Lx, yy = (si / Lx) % Ly, z = si / (Lx * Ly);
            auto site = [&](int64_t cx, int64_t cy, int64_t cz) {
                return cx + L.Lx * (cy + L.Ly * cz);
            };
            auto gather = [&](int64_t sn, float4* g) {
#pragma unroll
                for (int o = 0; o < B; ++o) g[o] = __ldg(u + (sn * B + o) * ldg + lane);
            };
            DFPair acc[B];
            float4 g[B];
            const double V =
                __dmul_rn(L.W, splitmix_uniform(L.seed, STREAM_DISORDER, (uint64_t)s) - 0.5);
            double up, lo;
            if (L.slab) {
                up = __dadd_rn(V, L.m);
                lo = __dadd_rn(V, -L.m);
            } else {
                up = __dadd_rn(L.m, V);
                lo = -up;
            }
            float up1, up2, lo1, lo2;
            df_split(up + shift, up1, up2);
            df_split(lo + shift, lo1, lo2);
            if constexpr (EXACT) {
                DFPair S[B];
                gather(site((x + L.Lx - 1) % L.Lx, yy, z), g);
                hop_sum_df<0>(S, g, 1.f, true);
                gather(site((x + 1) % L.Lx, yy, z), g);
                hop_sum_df<0>(S, g, -1.f, false);
                gather(site(x, (yy + L.Ly - 1) % L.Ly, z), g);
                hop_sum_df<1>(S, g, 1.f, false);
                gather(site(x, (yy + 1) % L.Ly, z), g);
                hop_sum_df<1>(S, g, -1.f, false);
                if (!L.slab || z > 0) {
                    gather(site(x, yy, (z + L.Lz - 1) % L.Lz), g);
                    hop_sum_df<2>(S, g, 1.f, false);
                }
                if (!L.slab || z + 1 < L.Lz) {
                    gather(site(x, yy, (z + 1) % L.Lz), g);
                    hop_sum_df<2>(S, g, -1.f, false);
                }
                gather(s, g);
#pragma unroll
                for (int o = 0; o < B; ++o) {
                    acc[o].hi = __fmul2_rn(make_float2(h1, h1), S[o].hi);
                    acc[o].lo = __fmul2_rn(make_float2(h1, h1), S[o].lo);
                    df_mac(acc[o], o < 2 ? up1 : lo1, o < 2 ? up2 : lo2, df_pair(g[o]));
                }
            } else {
#pragma unroll
                for (int r = 0; r < B; ++r) acc[r].hi = acc[r].lo = make_float2(0.f, 0.f);
                gather(s, g);
#pragma unroll
                for (int o = 0; o < B; ++o)
                    df_mac(acc[o], o < 2 ? up1 : lo1, o < 2 ? up2 : lo2, df_pair(g[o]));
                gather(site((x + L.Lx - 1) % L.Lx, yy, z), g);
                hop_df<0>(acc, g, h1, h2, 1.f);
                gather(site((x + 1) % L.Lx, yy, z), g);
                hop_df<0>(acc, g, h1, h2, -1.f);
                gather(site(x, (yy + L.Ly - 1) % L.Ly, z), g);
                hop_df<1>(acc, g, h1, h2, 1.f);
                gather(site(x, (yy + 1) % L.Ly, z), g);
                hop_df<1>(acc, g, h1, h2, -1.f);
                if (!L.slab || z > 0) {
                    gather(site(x, yy, (z + L.Lz - 1) % L.Lz), g);
                    hop_df<2>(acc, g, h1, h2, 1.f);
                }
                if (!L.slab || z + 1 < L.Lz) {
                    gather(site(x, yy, (z + 1) % L.Lz), g);
                    hop_df<2>(acc, g, h1, h2, -1.f);
                }
            }
#pragma unroll
            for (int r = 0; r < B; ++r) {
                const int64_t row = s * B + r;
                const DFPair hu = df_norm(acc[r]);
                const DFPair wo = df_pair(__ldcs(w + row * ldw + lane));
                DFPair wn;
                wn.hi = df_neg(wo.hi);
                wn.lo = df_neg(wo.lo);
                df_mac(wn, ta1, ta2, hu);  // 2 alpha (H + beta/alpha) u - w
                wn = df_norm(wn);
                DFPair yn = df_pair(__ldcs(y + row * ldy + lane));
                df_mac(yn, c1, c2, wn);
                yn = df_norm(yn);
                __stcs(w + row * ldw + lane, make_float4(wn.hi.x, wn.hi.y, wn.lo.x, wn.lo.y));
                __stcs(y + row * ldy + lane, make_float4(yn.hi.x, yn.hi.y, yn.lo.x, yn.lo.y));
            }
        }
        q = q_next;
        tt = tt + 1 == tile ? 0 : tt + 1;
    }
}

template <int G, int MINB, bool EXACT>
void launch_df_gm(const StencilView& v, const StepArgs& a, int wc, double shift, int sms,
                  cudaStream_t s) {
    auto kern = stencil_df_kernel<G, MINB, EXACT>;
    const int grid =
        sms * std::min(8, cached_occupancy(reinterpret_cast<const void*>(kern), ST_THREADS, 0));
    kern<<<grid, ST_THREADS, 0, s>>>(v, a, wc, shift);
}

// t/2 a power of two: no low word and every product by it exact.
bool exact_hopping(double hd) {
    int e = 0;
    return hd != 0.0 && std::fabs(std::frexp(hd, &e)) == 0.5 && e > -120 && e < 120;
}

// Resident CTAs per SM the register budget is fitted to (2, 3 or 4;
// CHEBFD_DF_FREE_CTAS overrides the default).
template <int G>
void launch_df_g(const StencilView& v, const StepArgs& a, int wc, double shift, int sms,
                 cudaStream_t s) {
    static const int minb = [] {
        const char* e = getenv("CHEBFD_DF_FREE_CTAS");
        return e ? std::min(4, std::max(2, atoi(e))) : 3;
    }();
    if (exact_hopping(v.hd)) {
        if (minb == 4)
            launch_df_gm<G, 4, true>(v, a, wc, shift, sms, s);
        else if (minb == 3)
            launch_df_gm<G, 3, true>(v, a, wc, shift, sms, s);
        else
            launch_df_gm<G, 2, true>(v, a, wc, shift, sms, s);
    } else {
        if (minb == 4)
            launch_df_gm<G, 4, false>(v, a, wc, shift, sms, s);
        else if (minb == 3)
            launch_df_gm<G, 3, false>(v, a, wc, shift, sms, s);
        else
            launch_df_gm<G, 2, false>(v, a, wc, shift, sms, s);
    }
}

StencilView view_of_gen(const Matrix& M) {
    StencilView v;
    v.Lx = M.gen.Lx;
    v.Ly = M.gen.Ly;
    v.Lz = M.gen.Lz;
    v.nsite = v.Lx * v.Ly * v.Lz;
    v.h = (float)(M.gen.t / 2.0);
    v.hd = M.gen.t / 2.0;
    v.m = M.gen.m;
    v.W = M.gen.W;
    v.seed = M.gen.seed;
    v.slab = M.gen.kind == CHEBFD_LATTICE_TOPI_SLAB ? 1 : 0;
    return v;
}

}  // namespace

// z-planes per CTA of the two-step kernel: a divisor of Lz, 8 preferred
// (halo overhead (Z + 2) / Z against enough CTAs); 0 if none fits.
int s2_planes(int64_t Lz) {
    for (int Z : {8, 10, 12, 16, 6, 5, 4})
        if (Lz % Z == 0) return Z;
    return Lz <= 16 ? (int)Lz : 0;
}

bool stencil2_applies(const Matrix& M, chebfd_dtype dt, int nb) {
    return M.stencil_pairs && M.stencil_enabled && M.has_gen && dt == CHEBFD_C64 &&
           nb == 2 * S2_WC &&
           M.gen.Lx % S2_TX == 0 && M.gen.Ly % S2_TY == 0 && s2_planes(M.gen.Lz) > 0 &&
           M.n < ((int64_t)1 << 31);
}

// Two fused Chebyshev steps on 16-column complex64 panels (ldw: the work
// panels' leading dimension in complex entries, ldy: the accumulated block's).
void launch_stencil2(const Matrix& M, const void* u0, const void* um, void* u1, void* u2,
                     void* y, int64_t ldw, int64_t ldy, double alpha, double beta, double c1,
                     double c2, cudaStream_t s) {
    const StencilView v = view_of_gen(M);
    S2Args a;
    a.u0 = (const float*)u0;
    a.um = (const float*)um;
    a.u1 = (float*)u1;
    a.u2 = (float*)u2;
    a.y = (float*)y;
    a.ldw = 2 * ldw;
    a.ldy = 2 * ldy;
    a.ta = (float)(2.0 * alpha);
    a.shift = (float)(beta / alpha);
    a.c1 = (float)c1;
    a.c2 = (float)c2;
    a.Z = s2_planes(v.Lz);
    ensure_dynamic_smem(reinterpret_cast<const void*>(stencil2_kernel), S2_RING_BYTES);
    const int grid = (int)((v.Lx / S2_TX) * (v.Ly / S2_TY) * (v.Lz / a.Z));
    stencil2_kernel<<<grid, S2_THREADS, S2_RING_BYTES, s>>>(v, a);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

bool stencil_step_applies(const Matrix& M, chebfd_dtype dt, StepMode mode, const StepArgs& a,
                          int wc) {
    return M.stencil_enabled && M.has_gen && dt == CHEBFD_C64 && mode == MODE_STEP &&
           a.moments == nullptr && a.coef == nullptr && wc >= 1 && wc <= 32;
}

void launch_stencil_step(const Matrix& M, const StepArgs& a, int wc, cudaStream_t s) {
    const StencilView v = view_of_gen(M);
    StepArgs b = a;
    static const int env_tile = [] {
        const char* e = getenv("CHEBFD_BELL_TILE");
        return e ? std::max(1, atoi(e)) : 1;
    }();
    b.tile = env_tile;
    const float shift = (float)(a.beta / a.alpha);
    if (wc > 16)
        launch_g<32>(v, b, wc, shift, M.num_sms, s);
    else if (wc > 8)
        launch_g<16>(v, b, wc, shift, M.num_sms, s);
    else if (wc > 4)
        launch_g<8>(v, b, wc, shift, M.num_sms, s);
    else
        launch_g<4>(v, b, wc, shift, M.num_sms, s);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

// Double-float matrix-free step (MODE_STEP) for the double-float filter.
bool stencil_df_applies(const Matrix& M, StepMode mode, int wc) {
    return M.stencil_enabled && M.has_gen && M.complex_values && mode == MODE_STEP && wc >= 1 &&
           wc <= 32;
}

void launch_stencil_df(const Matrix& M, const StepArgs& a, int wc, cudaStream_t s) {
    const StencilView v = view_of_gen(M);
    StepArgs b = a;
    b.tile = 1;
    b.order = site_order_of(M, wc);
    const double shift = a.beta / a.alpha;
    if (wc > 16)
        launch_df_g<32>(v, b, wc, shift, M.num_sms, s);
    else if (wc > 8)
        launch_df_g<16>(v, b, wc, shift, M.num_sms, s);
    else if (wc > 4)
        launch_df_g<8>(v, b, wc, shift, M.num_sms, s);
    else
        launch_df_g<4>(v, b, wc, shift, M.num_sms, s);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

}  // namespace chebfd
