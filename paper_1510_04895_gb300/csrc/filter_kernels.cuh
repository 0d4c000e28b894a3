// Fused Chebyshev step kernels (Fig. ChebFD, Sec. 4 "augmented spMMVM").
//
// One kernel launch performs one step of the filter recurrence for a block of
// nb row-major vectors in a single pass over the matrix and the vectors:
//   MODE_SPMV   : w = (alpha H + beta) u                       (also the first step)
//   MODE_SECOND : w = 2 (alpha H + beta) u - x ; x = c0 x + c1 u + c2 w
//   MODE_STEP   : w = 2 (alpha H + beta) u - w ; y = y + c0 w
// optionally with the per-column dot products <u,u>, <u,w> (SPMV: <u,u>,
// <u,w>) that give the Chebyshev moments of Sec. 4.
//
// Mapping: a group of G consecutive threads owns one matrix row (in SELL
// order); each thread owns CPT 16-byte chunks of the row's nb vector entries,
// so every gather of a neighbour row u_j is a contiguous, fully coalesced
// nb*S_v-byte segment read with 128-bit loads.  The row's column indices and
// values are read once per step for the whole block (broadcast inside the
// group).  Thread blocks are persistent and stride over the rows, so all SMs
// sweep the matrix as one front and the gathered rows of u are reused from L2.
#pragma once

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

template <class R, bool CPLX>
__device__ __forceinline__ void mac(ChunkT<R>& acc, const typename ValT<R, CPLX>::type& v,
                                    const ChunkT<R>& u) {
    constexpr int K = ChunkT<R>::K;
    if constexpr (CPLX) {
#pragma unroll
        for (int c = 0; c < K / 2; ++c) {
            const R ur = u.v[2 * c], ui = u.v[2 * c + 1];
            R ar = acc.v[2 * c], ai = acc.v[2 * c + 1];
            ar = fma(v.x, ur, ar);
            ar = fma(-v.y, ui, ar);
            ai = fma(v.x, ui, ai);
            ai = fma(v.y, ur, ai);
            acc.v[2 * c] = ar;
            acc.v[2 * c + 1] = ai;
        }
    } else {
#pragma unroll
        for (int c = 0; c < K; ++c) acc.v[c] = fma(v, u.v[c], acc.v[c]);
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
};

constexpr int STEP_THREADS = 256;

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

// Entries of one row handled per batch: all gathers of a batch are issued
// back to back (one memory latency per batch instead of one per entry).
template <int CPT>
struct Batch {
    static constexpr int EB = CPT == 1 ? 16 : 8;
};

template <class R, bool CPLX, int G, int CPT, int MODE>
__global__ void __launch_bounds__(STEP_THREADS, 2)
    cheb_step_kernel(SellView H, StepArgs a, int wc) {
    using V = typename ValT<R, CPLX>::type;
    using Chunk = ChunkT<R>;
    constexpr int K = Chunk::K;
    constexpr int CPC = CPLX ? K / 2 : K;  // vector columns per chunk
    constexpr int SLOTS = STEP_THREADS / G;
    constexpr int EB = Batch<CPT>::EB;
    constexpr int EPL = (EB + G - 1) / G;  // entries loaded per lane per batch
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

    const R alpha = (R)a.alpha, beta = (R)a.beta;
    const R two_alpha = (R)(2.0 * a.alpha), two_beta = (R)(2.0 * a.beta);
    const R c0 = (R)a.c0, c1 = (R)a.c1, c2 = (R)a.c2;

    R dot_a[CPT][CPC];
    R dot_b[CPT][CPC];
#pragma unroll
    for (int q = 0; q < CPT; ++q)
#pragma unroll
        for (int c = 0; c < CPC; ++c) dot_a[q][c] = dot_b[q][c] = (R)0;

    const int64_t nslots = (int64_t)gridDim.x * SLOTS;
    // Warp-uniform loop: every lane runs the same iterations so the shuffles
    // below always see the full warp; groups past the last row are inactive.
    for (int64_t r = (int64_t)blockIdx.x * SLOTS + slot; __any_sync(FULL, r < H.n); r += nslots) {
        const bool active = r < H.n;
        int64_t base = 0, orig = 0;
        int len = 0;
        if (active) {
            const int64_t k = r / H.C;
            base = __ldg(H.chunk_ptr + k) + (r - k * H.C);
            len = __ldg(H.chunk_len + k);
            orig = H.perm ? __ldg(H.perm + r) : r;
        }
        // own-row streams, issued before the gathers so their latency overlaps
        Chunk uo[CPT], xo[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int ci = lane + q * G;
            const bool on = active && ci < wc;
            const int64_t cofs = (int64_t)ci * K;
            if (on) uo[q] = load_chunk_ldg(u + orig * ldg + cofs);
            if (MODE == MODE_SECOND && on) xo[q] = load_chunk_cs(y + orig * ldy + cofs);
            if (MODE == MODE_STEP && on) xo[q] = load_chunk_cs(w + orig * ldw + cofs);
        }

        Chunk acc[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q)
#pragma unroll
            for (int c = 0; c < K; ++c) acc[q].v[c] = (R)0;

        const int maxlen = __reduce_max_sync(FULL, len);
        for (int j0 = 0; j0 < maxlen; j0 += EB) {
            // the group's lanes load the batch's column indices and values together
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
                    mc[e] = (int32_t)orig;
                    mv[e] = V{};
                }
            }
            // issue every gather of the batch, then accumulate
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
#pragma unroll
                        for (int c = 0; c < K; ++c) g[e][q].v[c] = (R)0;
                }
            }
#pragma unroll
            for (int e = 0; e < EB; ++e) {
                const V vj = shfl_val<R, CPLX>(mv[e / G], e % G, G);
#pragma unroll
                for (int q = 0; q < CPT; ++q) mac<R, CPLX>(acc[q], vj, g[e][q]);
            }
        }

#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int ci = lane + q * G;
            if (!active || ci >= wc) continue;
            const int64_t cofs = (int64_t)ci * K;
            R* wp = w + orig * ldw + cofs;
            R* yp = y + orig * ldy + cofs;
            Chunk wn;
            if (MODE == MODE_SPMV) {
#pragma unroll
                for (int c = 0; c < K; ++c) wn.v[c] = fma(alpha, acc[q].v[c], beta * uo[q].v[c]);
                store_chunk_cs(wp, wn);
            } else if (MODE == MODE_SECOND) {
                Chunk yn;
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    wn.v[c] = fma(two_alpha, acc[q].v[c], fma(two_beta, uo[q].v[c], -xo[q].v[c]));
                    yn.v[c] = fma(c2, wn.v[c], fma(c1, uo[q].v[c], c0 * xo[q].v[c]));
                }
                store_chunk_cs(wp, wn);
                store_chunk_cs(yp, yn);
            } else {
                const Chunk yo = load_chunk_cs(yp);
                Chunk yn;
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    wn.v[c] = fma(two_alpha, acc[q].v[c], fma(two_beta, uo[q].v[c], -xo[q].v[c]));
                    yn.v[c] = fma(c0, wn.v[c], yo.v[c]);
                }
                store_chunk_cs(wp, wn);
                store_chunk_cs(yp, yn);
            }
            if (dots) {
#pragma unroll
                for (int c = 0; c < CPC; ++c) {
                    if constexpr (CPLX) {
                        const R ur = uo[q].v[2 * c], ui = uo[q].v[2 * c + 1];
                        dot_a[q][c] = fma(ur, ur, fma(ui, ui, dot_a[q][c]));
                        dot_b[q][c] = fma(ur, wn.v[2 * c], fma(ui, wn.v[2 * c + 1], dot_b[q][c]));
                    } else {
                        dot_a[q][c] = fma(uo[q].v[c], uo[q].v[c], dot_a[q][c]);
                        dot_b[q][c] = fma(uo[q].v[c], wn.v[c], dot_b[q][c]);
                    }
                }
            }
        }
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
