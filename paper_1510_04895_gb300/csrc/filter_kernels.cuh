// Fused Chebyshev step kernels (Fig. ChebFD, Sec. 4 "augmented spMMVM").
//
// One kernel launch performs one step of the filter recurrence for a block of
// nb row-major vectors in a single pass over the matrix and the vectors:
//   MODE_SPMV   : w = (alpha H + beta) u                       (also the first step)
//   MODE_SECOND : w = 2 (alpha H + beta) u - x ; x = c0 x + c1 u + c2 w
//   MODE_STEP   : w = 2 (alpha H + beta) u - w ; y = y + c0 w
// optionally with the per-column dot products <u,u>, <u,w> that give the
// Chebyshev moments of Sec. 4.
//
// Mapping.  A group of G consecutive threads owns one matrix row (in SELL
// order); each thread owns CPT 16-byte chunks of the row's nb vector entries,
// so every gather of a neighbour row u_j is a contiguous, fully coalesced
// nb*S_v-byte read with 128-bit loads.  The row's column indices and values
// are loaded once per step for the whole block, cooperatively by the group,
// and broadcast with warp shuffles; all gathers of the row are then issued
// back to back.  All blocks sweep the rows as one front (a block takes a tile
// of consecutive row groups per wave), so the rows a lattice row gathers
// (same site, +-x neighbours) are mostly just read by the same block and hit
// in L1, and the far ones (+-y, +-z) were read by other SMs a moment earlier
// and hit in L2: u is read from DRAM about once per step.
//
// Fixed-width path (template L > 0): when every SELL chunk has the same width
// L (ELLPACK shape, no padding), row offsets need no metadata loads and the
// next row's indices/values are prefetched while the current row's gathers
// are in flight: one memory latency per row.  FP32 complex/real arithmetic
// uses the paired FMA of sm_100+ (__ffma2_rn).
#pragma once

#include <type_traits>

#include "common.cuh"

namespace chebfd {

template <class R>
struct ChunkT {
    static constexpr int K = 16 / sizeof(R);  // reals per 16-byte chunk
    R v[K];
};

template <class R>
__device__ __forceinline__ ChunkT<R> load_chunk_ldg(const R* p) {
    ChunkT<R> c;
    uint4 raw = __ldg(reinterpret_cast<const uint4*>(p));
    *reinterpret_cast<uint4*>(c.v) = raw;
    return c;
}
template <class R>
__device__ __forceinline__ ChunkT<R> load_chunk_cs(const R* p) {
    ChunkT<R> c;
    uint4 raw = __ldcs(reinterpret_cast<const uint4*>(p));
    *reinterpret_cast<uint4*>(c.v) = raw;
    return c;
}
template <class R>
__device__ __forceinline__ void store_chunk_cs(R* p, const ChunkT<R>& c) {
    __stcs(reinterpret_cast<uint4*>(p), *reinterpret_cast<const uint4*>(c.v));
}
template <class R>
__device__ __forceinline__ void zero_chunk(ChunkT<R>& c) {
#pragma unroll
    for (int i = 0; i < ChunkT<R>::K; ++i) c.v[i] = (R)0;
}

template <class R, bool CPLX>
struct ValT;
template <>
struct ValT<double, true> {
    using type = double2;
};
template <>
struct ValT<float, true> {
    using type = float2;
};
template <>
struct ValT<double, false> {
    using type = double;
};
template <>
struct ValT<float, false> {
    using type = float;
};

// Accumulator of one 16-byte chunk of sum_j H_ij u_j.  Complex values keep two
// partial sums, P = sum Re(h) (ur, ui) and Q = sum Im(h) (ur, ui); the complex
// product is formed once at the end, (P.x - Q.y, P.y + Q.x).  In FP32 each
// complex entry then costs two paired FMAs.
template <class R, bool CPLX>
struct Acc {
    ChunkT<R> p, q;
    __device__ __forceinline__ void zero() {
        zero_chunk(p);
        if (CPLX) zero_chunk(q);
    }
    __device__ __forceinline__ void mac(const typename ValT<R, CPLX>::type& h,
                                        const ChunkT<R>& u) {
        constexpr int K = ChunkT<R>::K;
        if constexpr (std::is_same<R, float>::value) {
            float2* P = reinterpret_cast<float2*>(p.v);
            float2* Q = reinterpret_cast<float2*>(q.v);
            const float2* U = reinterpret_cast<const float2*>(u.v);
            if constexpr (CPLX) {
                const float2 hr = make_float2(h.x, h.x), hi = make_float2(h.y, h.y);
#pragma unroll
                for (int c = 0; c < K / 2; ++c) {
                    P[c] = __ffma2_rn(hr, U[c], P[c]);
                    Q[c] = __ffma2_rn(hi, U[c], Q[c]);
                }
            } else {
                const float2 hh = make_float2(h, h);
#pragma unroll
                for (int c = 0; c < K / 2; ++c) P[c] = __ffma2_rn(hh, U[c], P[c]);
            }
        } else {
            if constexpr (CPLX) {
#pragma unroll
                for (int c = 0; c < K / 2; ++c) {
                    p.v[2 * c] = fma(h.x, u.v[2 * c], p.v[2 * c]);
                    p.v[2 * c + 1] = fma(h.x, u.v[2 * c + 1], p.v[2 * c + 1]);
                    q.v[2 * c] = fma(h.y, u.v[2 * c], q.v[2 * c]);
                    q.v[2 * c + 1] = fma(h.y, u.v[2 * c + 1], q.v[2 * c + 1]);
                }
            } else {
#pragma unroll
                for (int c = 0; c < K; ++c) p.v[c] = fma(h, u.v[c], p.v[c]);
            }
        }
    }
    __device__ __forceinline__ ChunkT<R> value() const {
        if constexpr (!CPLX) {
            return p;
        } else {
            ChunkT<R> r;
#pragma unroll
            for (int c = 0; c < ChunkT<R>::K / 2; ++c) {
                r.v[2 * c] = p.v[2 * c] - q.v[2 * c + 1];
                r.v[2 * c + 1] = p.v[2 * c + 1] + q.v[2 * c];
            }
            return r;
        }
    }
};

// d = a * x + y on chunks (paired FMA for FP32).
template <class R>
__device__ __forceinline__ ChunkT<R> axpy_chunk(R a, const ChunkT<R>& x, const ChunkT<R>& y) {
    ChunkT<R> d;
    if constexpr (std::is_same<R, float>::value) {
        const float2 aa = make_float2(a, a);
        const float2* X = reinterpret_cast<const float2*>(x.v);
        const float2* Y = reinterpret_cast<const float2*>(y.v);
        float2* D = reinterpret_cast<float2*>(d.v);
#pragma unroll
        for (int c = 0; c < ChunkT<R>::K / 2; ++c) D[c] = __ffma2_rn(aa, X[c], Y[c]);
    } else {
#pragma unroll
        for (int c = 0; c < ChunkT<R>::K; ++c) d.v[c] = fma(a, x.v[c], y.v[c]);
    }
    return d;
}

template <class R>
__device__ __forceinline__ ChunkT<R> scale_chunk(R a, const ChunkT<R>& x) {
    ChunkT<R> d;
#pragma unroll
    for (int c = 0; c < ChunkT<R>::K; ++c) d.v[c] = a * x.v[c];
    return d;
}

template <class R>
__device__ __forceinline__ ChunkT<R> neg_chunk(const ChunkT<R>& x) {
    ChunkT<R> d;
#pragma unroll
    for (int c = 0; c < ChunkT<R>::K; ++c) d.v[c] = -x.v[c];
    return d;
}

template <class R, bool CPLX>
__device__ __forceinline__ typename ValT<R, CPLX>::type shfl_val(
    const typename ValT<R, CPLX>::type& v, int src, int width) {
    if constexpr (CPLX) {
        typename ValT<R, CPLX>::type o;
        o.x = __shfl_sync(0xffffffffu, v.x, src, width);
        o.y = __shfl_sync(0xffffffffu, v.y, src, width);
        return o;
    } else {
        return __shfl_sync(0xffffffffu, v, src, width);
    }
}

struct SellView {
    const int64_t* chunk_ptr;
    const int32_t* chunk_len;
    const int32_t* col;
    const void* val;
    const int64_t* perm;  // nullptr when identity
    int64_t n;
    int C;
    int logC;  // C is a power of two: chunk of row r = r >> logC
};

constexpr int STEP_THREADS = 256;

// Entries of one row handled per batch on the generic (variable-width) path.
template <int CPT>
struct Batch {
    static constexpr int EB = CPT == 1 ? 16 : 8;
};

// ENS: rows of an ensemble read their member's alpha, beta and g_n c_n from a
// coefficient table (a separate instantiation, so the single-matrix kernel
// carries none of that code).
template <class R, bool CPLX, int G, int CPT, int MODE, int L, bool ENS>
__global__ void __launch_bounds__(STEP_THREADS, sizeof(R) == 4 ? 3 : 2)
    cheb_step_kernel(SellView H, StepArgs a, int wc) {
    using V = typename ValT<R, CPLX>::type;
    using Chunk = ChunkT<R>;
    constexpr int K = Chunk::K;
    constexpr int CPC = CPLX ? K / 2 : K;  // vector columns per chunk
    constexpr int SLOTS = STEP_THREADS / G;
    constexpr int EB = L > 0 ? L : Batch<CPT>::EB;  // entries per batch
    constexpr int EPL = (EB + G - 1) / G;           // entries loaded per lane per batch
    constexpr unsigned FULL = 0xffffffffu;

    const V* __restrict__ val = reinterpret_cast<const V*>(H.val);
    const int32_t* __restrict__ colp = H.col;
    const R* __restrict__ u = reinterpret_cast<const R*>(a.gather);
    R* __restrict__ w = reinterpret_cast<R*>(a.w);
    R* __restrict__ y = reinterpret_cast<R*>(a.y);

    const int lane = threadIdx.x % G;
    const int slot = threadIdx.x / G;
    const bool dots = a.moments != nullptr;
    constexpr int RPE = CPLX ? 2 : 1;  // reals per vector element
    const int64_t ldg = a.ldg * RPE, ldw = a.ldw * RPE, ldy = a.ldy * RPE;

    // per-launch scalars (an ensemble row overwrites them with its member's)
    R alpha = (R)a.alpha, beta = (R)a.beta;
    R two_alpha = (R)(2.0 * a.alpha), two_beta = (R)(2.0 * a.beta);
    R c0 = (R)a.c0, c1 = (R)a.c1, c2 = (R)a.c2;

    R dot_a[CPT][CPC];
    R dot_b[CPT][CPC];
#pragma unroll
    for (int q = 0; q < CPT; ++q)
#pragma unroll
        for (int c = 0; c < CPC; ++c) dot_a[q][c] = dot_b[q][c] = (R)0;

    // Row order: all blocks sweep the matrix as one front.  In wave w, block b
    // takes the `tile` consecutive row groups starting at (w*grid + b)*tile*SLOTS,
    // so a row's far neighbours (lattice +-z) are read by other SMs within one
    // or two waves and stay in L2, while neighbours inside the tile hit in L1.
    // The trip count is block-uniform, so every lane runs every iteration and
    // the shuffles see the full warp.
    const int tile = a.tile > 0 ? a.tile : 1;
    const int64_t wave_rows = (int64_t)gridDim.x * tile * SLOTS;
    const int iters = (int)((H.n + wave_rows - 1) / wave_rows) * tile;
    const int64_t r_end = H.n;
    const int64_t cmask = H.C - 1;
    // row of iteration it = (wave w, tile step t): advanced incrementally, so
    // the loop carries no integer division
    const int64_t wrap = wave_rows - (int64_t)(tile - 1) * SLOTS;
    auto advance = [&](int64_t rr, int t) -> int64_t { return t + 1 == tile ? rr + wrap : rr + SLOTS; };
    int64_t r = (int64_t)blockIdx.x * tile * SLOTS + slot;
    int t_in_tile = 0;

    // Fixed-width path: the next row's entries are prefetched into (nc, nv).
    int32_t nc[EPL];
    V nv[EPL];
    auto load_entries = [&](int64_t rr) {
        const bool act = rr < r_end;
        const int64_t k = rr >> H.logC;
        const int64_t base = (k << H.logC) * L + (rr & cmask);
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
            const int j = lane + e * G;
            if (act && j < L) {
                const int64_t pos = base + (int64_t)j * H.C;
                nc[e] = __ldcs(colp + pos);
                nv[e] = __ldcs(val + pos);
            } else {
                nc[e] = 0;
                nv[e] = V{};
            }
        }
    };
    if constexpr (L > 0) load_entries(r);

    for (int it = 0; it < iters; ++it) {
        const int64_t r_next = advance(r, t_in_tile);
        const bool active = r < r_end;
        const int64_t orig = active ? (H.perm ? __ldg(H.perm + r) : r) : 0;

        // ensemble: this row's member coefficients (tiny table, L1-resident)
        if constexpr (ENS) {
            if (active) {
                const double* cf = a.coef + (int64_t)__ldg(a.row_inst + orig) * a.coef_ld;
                const double al = __ldg(cf), be = __ldg(cf + 1);
                alpha = (R)al;
                beta = (R)be;
                two_alpha = (R)(2.0 * al);
                two_beta = (R)(2.0 * be);
                if (MODE == MODE_SECOND) {
                    c0 = (R)__ldg(cf + 2);
                    c1 = (R)__ldg(cf + 3);
                    c2 = (R)__ldg(cf + 4);
                } else if (MODE == MODE_STEP) {
                    c0 = (R)__ldg(cf + 2 + a.mom_step);
                }
            }
        }

        // own-row streams, issued before the gathers so their latency overlaps
        Chunk uo[CPT], xo[CPT], yo[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int ci = lane + q * G;
            const bool on = active && ci < wc;
            const int64_t cofs = (int64_t)ci * K;
            if (on) uo[q] = load_chunk_ldg(u + orig * ldg + cofs);
            if (MODE == MODE_SECOND && on) xo[q] = load_chunk_cs(y + orig * ldy + cofs);
            if (MODE == MODE_STEP && on) {
                xo[q] = load_chunk_cs(w + orig * ldw + cofs);
                yo[q] = load_chunk_cs(y + orig * ldy + cofs);
            }
        }

        Acc<R, CPLX> acc[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q) acc[q].zero();

        if constexpr (L > 0) {
            int32_t mc[EPL];
            V mv[EPL];
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
                mc[e] = nc[e];
                mv[e] = nv[e];
            }
            // gathers of this row
            Chunk g[L][CPT];
#pragma unroll
            for (int e = 0; e < L; ++e) {
                const int cj = __shfl_sync(FULL, mc[e / G], e % G, G);
                const R* urow = u + (int64_t)cj * ldg;
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    const int ci = lane + q * G;
                    if (active && ci < wc)
                        g[e][q] = load_chunk_ldg(urow + (int64_t)ci * K);
                    else
                        zero_chunk(g[e][q]);
                }
            }
            // prefetch the next row's entries while the gathers are in flight
            load_entries(r_next);
#pragma unroll
            for (int e = 0; e < L; ++e) {
                const V vj = shfl_val<R, CPLX>(mv[e / G], e % G, G);
#pragma unroll
                for (int q = 0; q < CPT; ++q) acc[q].mac(vj, g[e][q]);
            }
        } else {
            int64_t base = 0;
            int len = 0;
            if (active) {
                const int64_t k = r >> H.logC;
                base = __ldg(H.chunk_ptr + k) + (r & cmask);
                len = __ldg(H.chunk_len + k);
            }
            const int maxlen = __reduce_max_sync(FULL, len);
            for (int j0 = 0; j0 < maxlen; j0 += EB) {
                int32_t mc[EPL];
                V mv[EPL];
#pragma unroll
                for (int e = 0; e < EPL; ++e) {
                    const int j = j0 + lane + e * G;
                    if (j < len) {
                        const int64_t pos = base + (int64_t)j * H.C;
                        mc[e] = __ldcs(colp + pos);
                        mv[e] = __ldcs(val + pos);
                    } else {
                        mc[e] = 0;
                        mv[e] = V{};
                    }
                }
                Chunk g[EB][CPT];
#pragma unroll
                for (int e = 0; e < EB; ++e) {
                    const int cj = __shfl_sync(FULL, mc[e / G], e % G, G);
                    const R* urow = u + (int64_t)cj * ldg;
#pragma unroll
                    for (int q = 0; q < CPT; ++q) {
                        const int ci = lane + q * G;
                        if (j0 + e < len && ci < wc)
                            g[e][q] = load_chunk_ldg(urow + (int64_t)ci * K);
                        else
                            zero_chunk(g[e][q]);
                    }
                }
#pragma unroll
                for (int e = 0; e < EB; ++e) {
                    const V vj = shfl_val<R, CPLX>(mv[e / G], e % G, G);
#pragma unroll
                    for (int q = 0; q < CPT; ++q) acc[q].mac(vj, g[e][q]);
                }
            }
        }

#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int ci = lane + q * G;
            if (!active || ci >= wc) continue;
            const int64_t cofs = (int64_t)ci * K;
            R* wp = w + orig * ldw + cofs;
            R* yp = y + orig * ldy + cofs;
            const Chunk hu = acc[q].value();  // (H u)_i
            Chunk wn;
            if (MODE == MODE_SPMV) {
                wn = axpy_chunk(alpha, hu, scale_chunk(beta, uo[q]));
                store_chunk_cs(wp, wn);
            } else if (MODE == MODE_SECOND) {
                // w = 2 alpha Hu + (2 beta u - x) ; y = c2 w + (c1 u + c0 x)
                wn = axpy_chunk(two_alpha, hu, axpy_chunk(two_beta, uo[q], neg_chunk(xo[q])));
                const Chunk yn =
                    axpy_chunk(c2, wn, axpy_chunk(c1, uo[q], scale_chunk(c0, xo[q])));
                store_chunk_cs(wp, wn);
                store_chunk_cs(yp, yn);
            } else {
                wn = axpy_chunk(two_alpha, hu, axpy_chunk(two_beta, uo[q], neg_chunk(xo[q])));
                const Chunk yn = axpy_chunk(c0, wn, yo[q]);
                store_chunk_cs(wp, wn);
                store_chunk_cs(yp, yn);
            }
            if (dots) {
#pragma unroll
                for (int c = 0; c < CPC; ++c) {
                    if constexpr (CPLX) {
                        const R ur = uo[q].v[2 * c], ui = uo[q].v[2 * c + 1];
                        dot_a[q][c] = fma(ur, ur, fma(ui, ui, dot_a[q][c]));
                        dot_b[q][c] =
                            fma(ur, wn.v[2 * c], fma(ui, wn.v[2 * c + 1], dot_b[q][c]));
                    } else {
                        dot_a[q][c] = fma(uo[q].v[c], uo[q].v[c], dot_a[q][c]);
                        dot_b[q][c] = fma(uo[q].v[c], wn.v[c], dot_b[q][c]);
                    }
                }
            }
        }
        r = r_next;
        t_in_tile = t_in_tile + 1 == tile ? 0 : t_in_tile + 1;
    }

    if (!dots) return;

    // ---- deterministic reduction of the per-column dots -----------------------
    // 1. per block: slots summed in a fixed order through shared memory;
    // 2. per grid: the last block to finish sums the block partials in block order.
    extern __shared__ double smem[];  // [SLOTS][2][nb]
    const int nb = a.nb;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int ci = lane + q * G;
        if (ci >= wc) continue;
#pragma unroll
        for (int c = 0; c < CPC; ++c) {
            const int col = ci * CPC + c;
            smem[(slot * 2 + 0) * nb + col] = (double)dot_a[q][c];
            smem[(slot * 2 + 1) * nb + col] = (double)dot_b[q][c];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * nb; t += blockDim.x) {
        double s = 0.0;
        for (int sl = 0; sl < SLOTS; ++sl) s += smem[sl * 2 * nb + t];
        a.partials[(int64_t)blockIdx.x * 2 * nb + t] = s;
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned int is_last;
    if (threadIdx.x == 0) is_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int t = threadIdx.x; t < 2 * nb; t += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b)
            s += __ldcg(a.partials + (int64_t)b * 2 * nb + t);
        const int which = t / nb, col = t % nb;
        double* mom = a.moments;
        if (MODE == MODE_SPMV) {
            // <x,x> = mu_0, <x, A x> = mu_1
            mom[(int64_t)which * a.mom_ld + col] = s;
        } else {
            const int n = a.mom_step;
            const int64_t row = which == 0 ? 2 * n - 2 : 2 * n - 1;
            const double base = mom[(int64_t)which * a.mom_ld + col];  // mu_0 or mu_1
            mom[row * a.mom_ld + col] = 2.0 * s - base;
        }
    }
    if (threadIdx.x == 0) *a.counter = 0u;
}

}  // namespace chebfd
