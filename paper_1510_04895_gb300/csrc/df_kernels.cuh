// Fused Chebyshev step in double-float arithmetic (the FP64-class sweep of
// the mixed-precision solve, Fig. ChebFD modes SPMV / SECOND / STEP).
//
// GB300 executes FP64 at ~1/64 of its FP32 rate, so the FP64 filter is
// ALU-bound at ~1.1 TFLOP/s.  Here every vector entry and matrix value is a
// double-float (hi + lo floats, 48-bit significand) and all arithmetic runs
// on the paired FP32 pipe (df.cuh): one 16-byte chunk holds one complex
// entry (re/im pairs) or two real entries, the same bytes per entry as FP64.
// The mapping follows the FP32 step kernel: G lanes per row, lane = chunk,
// column indices loaded cooperatively and broadcast by shuffles, fixed-width
// rows (L = 13 insulator, 4 graphene) prefetch the next row's entries while
// the gathers are in flight, persistent grid in wave-front row order.
#pragma once

#include "df.cuh"
#include "filter_kernels.cuh"

namespace chebfd {

template <bool CPLX>
struct DFVal;
template <>
struct DFVal<true> {
    using type = float4;  // (re_hi, re_lo, im_hi, im_lo)
};
template <>
struct DFVal<false> {
    using type = float2;  // (hi, lo)
};

__device__ __forceinline__ DFPair df_of(const float4& c) {
    DFPair p;
    p.hi = make_float2(c.x, c.y);
    p.lo = make_float2(c.z, c.w);
    return p;
}
__device__ __forceinline__ float4 df_pack(const DFPair& p) {
    return make_float4(p.hi.x, p.hi.y, p.lo.x, p.lo.y);
}

__device__ __forceinline__ float4 shfl_dfval(const float4& v, int src, int width) {
    return make_float4(__shfl_sync(0xffffffffu, v.x, src, width),
                       __shfl_sync(0xffffffffu, v.y, src, width),
                       __shfl_sync(0xffffffffu, v.z, src, width),
                       __shfl_sync(0xffffffffu, v.w, src, width));
}
__device__ __forceinline__ float2 shfl_dfval(const float2& v, int src, int width) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src, width),
                       __shfl_sync(0xffffffffu, v.y, src, width));
}

// Product of one row with a chunk: P = sum h_re * u, Q = sum h_im * u (complex),
// combined at the end as (P.re - Q.im, P.im + Q.re).
template <bool CPLX>
struct DFAcc {
    DFPair P, Q;
    __device__ __forceinline__ void zero() {
        P.hi = P.lo = Q.hi = Q.lo = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void mac(const typename DFVal<CPLX>::type& h, const DFPair& u) {
        if constexpr (CPLX) {
            df_mac(P, h.x, h.y, u);
            df_mac(Q, h.z, h.w, u);
        } else {
            df_mac(P, h.x, h.y, u);
        }
    }
    __device__ __forceinline__ DFPair value() const {
        if constexpr (CPLX) {
            DFPair r = P, q;
            q.hi = make_float2(-Q.hi.y, Q.hi.x);
            q.lo = make_float2(-Q.lo.y, Q.lo.x);
            df_add(r, q);
            return df_norm(r);
        } else {
            return df_norm(P);
        }
    }
};

// a.ldg / a.ldw / a.ldy are row strides in 16-byte chunks.
template <bool CPLX, int G, int MODE, int L>
__global__ void __launch_bounds__(STEP_THREADS, 2)
    cheb_df_kernel(SellView H, StepArgs a, int wc) {
    using V = typename DFVal<CPLX>::type;
    constexpr int SLOTS = STEP_THREADS / G;
    constexpr int EB = L > 0 ? L : 8;
    constexpr int EPL = (EB + G - 1) / G;
    constexpr unsigned FULL = 0xffffffffu;

    const V* __restrict__ val = reinterpret_cast<const V*>(H.val);
    const int32_t* __restrict__ colp = H.col;
    const float4* __restrict__ u = reinterpret_cast<const float4*>(a.gather);
    float4* __restrict__ w = reinterpret_cast<float4*>(a.w);
    float4* __restrict__ y = reinterpret_cast<float4*>(a.y);
    const int lane = threadIdx.x % G;
    const int slot = threadIdx.x / G;
    const bool on = lane < wc;
    const int64_t ldg = a.ldg, ldw = a.ldw, ldy = a.ldy;

    // scalars as double-floats
    float s_a1, s_a2, s_b1, s_b2, c01, c02, c11, c12, c21, c22;
    const double amul = MODE == MODE_SPMV ? 1.0 : 2.0;
    df_split(amul * a.alpha, s_a1, s_a2);
    df_split(amul * a.beta, s_b1, s_b2);
    df_split(a.c0, c01, c02);
    df_split(a.c1, c11, c12);
    df_split(a.c2, c21, c22);

    const int tile = a.tile > 0 ? a.tile : 1;
    const int64_t wave_rows = (int64_t)gridDim.x * tile * SLOTS;
    const int iters = (int)((H.n + wave_rows - 1) / wave_rows) * tile;
    const int64_t r_end = H.n;
    const int64_t cmask = H.C - 1;
    const int64_t wrap = wave_rows - (int64_t)(tile - 1) * SLOTS;
    int64_t r = (int64_t)blockIdx.x * tile * SLOTS + slot;
    int t_in_tile = 0;

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
        const int64_t r_next = t_in_tile + 1 == tile ? r + wrap : r + SLOTS;
        const bool active = r < r_end;
        const int64_t orig = active ? (H.perm ? __ldg(H.perm + r) : r) : 0;
        const bool mine = active && on;

        float4 uo = make_float4(0.f, 0.f, 0.f, 0.f), xo = uo, yo = uo;
        if (mine) {
            uo = __ldg(u + orig * ldg + lane);
            if (MODE == MODE_SECOND) xo = __ldcs(y + orig * ldy + lane);
            if (MODE == MODE_STEP) {
                xo = __ldcs(w + orig * ldw + lane);
                yo = __ldcs(y + orig * ldy + lane);
            }
        }

        DFAcc<CPLX> acc;
        acc.zero();
        if constexpr (L > 0) {
            int32_t mc[EPL];
            V mv[EPL];
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
                mc[e] = nc[e];
                mv[e] = nv[e];
            }
            float4 g[L];
#pragma unroll
            for (int e = 0; e < L; ++e) {
                const int cj = __shfl_sync(FULL, mc[e / G], e % G, G);
                g[e] = mine ? __ldg(u + (int64_t)cj * ldg + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            load_entries(r_next);
#pragma unroll
            for (int e = 0; e < L; ++e) acc.mac(shfl_dfval(mv[e / G], e % G, G), df_of(g[e]));
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
                float4 g[EB];
#pragma unroll
                for (int e = 0; e < EB; ++e) {
                    const int cj = __shfl_sync(FULL, mc[e / G], e % G, G);
                    g[e] = (mine && j0 + e < len) ? __ldg(u + (int64_t)cj * ldg + lane)
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int e = 0; e < EB; ++e)
                    acc.mac(shfl_dfval(mv[e / G], e % G, G), df_of(g[e]));
            }
        }

        if (mine) {
            const DFPair hu = acc.value();
            const DFPair U = df_of(uo);
            DFPair wn;
            if (MODE == MODE_SPMV) {
                wn.hi = wn.lo = make_float2(0.f, 0.f);
                df_mac(wn, s_a1, s_a2, hu);
                df_mac(wn, s_b1, s_b2, U);
                wn = df_norm(wn);
                w[orig * ldw + lane] = df_pack(wn);
            } else {
                // w = 2 alpha Hu + 2 beta u - x
                const DFPair X = df_of(xo);
                wn.hi = df_neg(X.hi);
                wn.lo = df_neg(X.lo);
                df_mac(wn, s_a1, s_a2, hu);
                df_mac(wn, s_b1, s_b2, U);
                wn = df_norm(wn);
                DFPair yn;
                if (MODE == MODE_SECOND) {
                    // y = c0 x + c1 u + c2 w
                    yn.hi = yn.lo = make_float2(0.f, 0.f);
                    df_mac(yn, c01, c02, X);
                    df_mac(yn, c11, c12, U);
                    df_mac(yn, c21, c22, wn);
                } else {
                    // y = y + c w
                    yn = df_of(yo);
                    df_mac(yn, c01, c02, wn);
                }
                yn = df_norm(yn);
                __stcs(w + orig * ldw + lane, df_pack(wn));
                __stcs(y + orig * ldy + lane, df_pack(yn));
            }
        }
        r = r_next;
        t_in_tile = t_in_tile + 1 == tile ? 0 : t_in_tile + 1;
    }
}

}  // namespace chebfd
