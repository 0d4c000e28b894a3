// Tall-skinny products of the dense steps (Sec. 3.1 steps 6-7) in
// double-float arithmetic on the paired FP32 pipe (df.cuh), for the MIXED_DF
// solve: GB300's FP64 GEMM runs at ~1.1 TFLOP/s, the same contraction in
// double-float on the FP32 pipe several times faster.  Inputs and outputs
// stay FP64 (split into hi + lo floats while staging tiles in shared memory,
// summed back on output); unit roundoff ~2^-48.
//
//   df_gram: C (m x m, column-major) = sum_k A[k][i] conj(B[k][j])
//            (A, B: row-major n x m blocks; the convention of gemm_nh)
//   df_gemm: T[p][i] = sum_q Y[p][q] conj(M(q, i))
//            (Y row-major n x k, M column-major k x r; the convention of gemm_ch)
//
// Complex products a conj(b) use P = b_re (a_re, a_im), Q = b_im (a_re, a_im):
// a conj(b) = (P.re + Q.im, P.im - Q.re).  The Gram is split over row chunks;
// each chunk's partial tile is written as double-float and the partials are
// summed in chunk order (deterministic).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "df.cuh"

namespace chebfd {

namespace {

constexpr int GT = 32;        // Gram output tile (GT x GT) per block
constexpr int GR = 32;        // rows staged per step
constexpr int DF_THREADS = 256;

struct DFC {  // one complex double-float: hi = (re, im), lo = (re, im)
    float2 hi, lo;
};

__device__ __forceinline__ DFC split_c(const double* p) {
    DFC r;
    df_split(p[0], r.hi.x, r.lo.x);
    df_split(p[1], r.hi.y, r.lo.y);
    return r;
}
__device__ __forceinline__ float2 split_r(double v) {
    float2 r;
    df_split(v, r.x, r.y);
    return r;
}

// acc_P += b_re * a, acc_Q += b_im * a  (a, b complex double-float)
__device__ __forceinline__ void mac_conj(DFPair& P, DFPair& Q, const DFC& a, const DFC& b) {
    DFPair av;
    av.hi = a.hi;
    av.lo = a.lo;
    df_mac(P, b.hi.x, b.lo.x, av);
    df_mac(Q, b.hi.y, b.lo.y, av);
}

__device__ __forceinline__ DFPair conj_result(const DFPair& P, const DFPair& Q) {
    DFPair r = P, q;
    q.hi = make_float2(Q.hi.y, -Q.hi.x);
    q.lo = make_float2(Q.lo.y, -Q.lo.x);
    df_add(r, q);
    return df_norm(r);
}

__device__ __forceinline__ void zero(DFPair& p) { p.hi = p.lo = make_float2(0.f, 0.f); }

// Complex Gram, one GT x GT tile of C per block and one row chunk per blockIdx.y.
// Thread (ty, tx) owns outputs (i0 + 2 ty + {0,1}, j0 + 2 tx + {0,1}).
__global__ void __launch_bounds__(DF_THREADS)
    df_gram_c_kernel(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n,
                     int m, int64_t rows_per_chunk, int tiles_j, float4* partial) {
    __shared__ DFC As[GR][GT];
    __shared__ DFC Bs[GR][GT];
    const int ti = blockIdx.x / tiles_j, tj = blockIdx.x % tiles_j;
    const int i0 = ti * GT, j0 = tj * GT;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const int64_t k_beg = blockIdx.y * rows_per_chunk;
    const int64_t k_end = min(n, k_beg + rows_per_chunk);
    DFPair P[2][2], Q[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            zero(P[a][b]);
            zero(Q[a][b]);
        }
    int step = 0;
    for (int64_t k0 = k_beg; k0 < k_end; k0 += GR, ++step) {
        for (int e = threadIdx.x; e < GR * GT; e += DF_THREADS) {
            const int r = e / GT, c = e % GT;
            const int64_t k = k0 + r;
            const bool in = k < k_end;
            DFC za;
            za.hi = za.lo = make_float2(0.f, 0.f);
            As[r][c] = (in && i0 + c < m) ? split_c(A + 2 * (k * lda + i0 + c)) : za;
            Bs[r][c] = (in && j0 + c < m) ? split_c(B + 2 * (k * ldb + j0 + c)) : za;
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < GR; ++r) {
            const DFC a0 = As[r][2 * ty], a1 = As[r][2 * ty + 1];
            const DFC b0 = Bs[r][2 * tx], b1 = Bs[r][2 * tx + 1];
            mac_conj(P[0][0], Q[0][0], a0, b0);
            mac_conj(P[0][1], Q[0][1], a0, b1);
            mac_conj(P[1][0], Q[1][0], a1, b0);
            mac_conj(P[1][1], Q[1][1], a1, b1);
        }
        __syncthreads();
        if ((step & 7) == 7) {  // keep the low parts small
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    P[a][b] = df_norm(P[a][b]);
                    Q[a][b] = df_norm(Q[a][b]);
                }
        }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = i0 + 2 * ty + a, j = j0 + 2 * tx + b;
            if (i < m && j < m) {
                const DFPair v = conj_result(P[a][b], Q[a][b]);
                partial[(int64_t)blockIdx.y * m * m + (int64_t)j * m + i] =
                    make_float4(v.hi.x, v.hi.y, v.lo.x, v.lo.y);
            }
        }
}

// Real Gram: thread (ty, tx) owns (i0 + 2 ty + {0,1}) x (j0 + 2 tx + {0,1}),
// the two i's of a j paired in one double-float pair.
__global__ void __launch_bounds__(DF_THREADS)
    df_gram_r_kernel(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n,
                     int m, int64_t rows_per_chunk, int tiles_j, float4* partial) {
    __shared__ float2 As[GR][GT];
    __shared__ float2 Bs[GR][GT];
    const int ti = blockIdx.x / tiles_j, tj = blockIdx.x % tiles_j;
    const int i0 = ti * GT, j0 = tj * GT;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const int64_t k_beg = blockIdx.y * rows_per_chunk;
    const int64_t k_end = min(n, k_beg + rows_per_chunk);
    DFPair S[2];
    zero(S[0]);
    zero(S[1]);
    int step = 0;
    for (int64_t k0 = k_beg; k0 < k_end; k0 += GR, ++step) {
        for (int e = threadIdx.x; e < GR * GT; e += DF_THREADS) {
            const int r = e / GT, c = e % GT;
            const int64_t k = k0 + r;
            const bool in = k < k_end;
            As[r][c] = (in && i0 + c < m) ? split_r(A[k * lda + i0 + c]) : make_float2(0.f, 0.f);
            Bs[r][c] = (in && j0 + c < m) ? split_r(B[k * ldb + j0 + c]) : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < GR; ++r) {
            const float2 a0 = As[r][2 * ty], a1 = As[r][2 * ty + 1];
            DFPair av;
            av.hi = make_float2(a0.x, a1.x);
            av.lo = make_float2(a0.y, a1.y);
            const float2 b0 = Bs[r][2 * tx], b1 = Bs[r][2 * tx + 1];
            df_mac(S[0], b0.x, b0.y, av);
            df_mac(S[1], b1.x, b1.y, av);
        }
        __syncthreads();
        if ((step & 7) == 7) {
            S[0] = df_norm(S[0]);
            S[1] = df_norm(S[1]);
        }
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const DFPair v = df_norm(S[b]);
        const int j = j0 + 2 * tx + b;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int i = i0 + 2 * ty + a;
            if (i < m && j < m)
                partial[(int64_t)blockIdx.y * m * m + (int64_t)j * m + i] =
                    make_float4(a ? v.hi.y : v.hi.x, 0.f, a ? v.lo.y : v.lo.x, 0.f);
        }
    }
}

// C (column-major m x m, FP64) = sum over chunks, in chunk order.
template <bool CPLX>
__global__ void df_gram_reduce_kernel(const float4* partial, int chunks, int m, double* C) {
    const int64_t mm = (int64_t)m * m;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < mm;
         t += (int64_t)gridDim.x * blockDim.x) {
        DFPair s;
        zero(s);
        for (int c = 0; c < chunks; ++c) {
            const float4 v = partial[c * mm + t];
            DFPair p;
            p.hi = make_float2(v.x, v.y);
            p.lo = make_float2(v.z, v.w);
            df_add(s, p);
        }
        s = df_norm(s);
        if (CPLX) {
            C[2 * t] = (double)s.hi.x + (double)s.lo.x;
            C[2 * t + 1] = (double)s.hi.y + (double)s.lo.y;
        } else {
            C[t] = (double)s.hi.x + (double)s.lo.x;
        }
    }
}

constexpr int MP = 64;  // rows of T per block
constexpr int MI = 32;  // columns of T per block
constexpr int MQ = 16;  // inner dimension staged per step

// T[p][i] = sum_q Y[p][q] conj(M(q, i)); thread (tp, tc) owns rows
// p0 + 2 tp + {0,1} and columns i0 + 4 tc + {0..3}.
__global__ void __launch_bounds__(DF_THREADS)
    df_gemm_c_kernel(const double* Mt, int ldm, const double* Y, int64_t ldy, int64_t n, int k,
                     int r, double* T, int64_t ldt) {
    __shared__ DFC Ys[MP][MQ];
    __shared__ DFC Ms[MQ][MI];
    const int64_t p0 = (int64_t)blockIdx.x * MP;
    const int i0 = blockIdx.y * MI;
    const int tp = threadIdx.x / 8, tc = threadIdx.x % 8;
    DFPair P[2][4], Q[2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            zero(P[a][b]);
            zero(Q[a][b]);
        }
    DFC za;
    za.hi = za.lo = make_float2(0.f, 0.f);
    for (int q0 = 0; q0 < k; q0 += MQ) {
        for (int e = threadIdx.x; e < MP * MQ; e += DF_THREADS) {
            const int rr = e / MQ, c = e % MQ;
            const int64_t p = p0 + rr;
            Ys[rr][c] = (p < n && q0 + c < k) ? split_c(Y + 2 * (p * ldy + q0 + c)) : za;
        }
        for (int e = threadIdx.x; e < MQ * MI; e += DF_THREADS) {
            const int q = e / MI, c = e % MI;
            Ms[q][c] = (q0 + q < k && i0 + c < r) ? split_c(Mt + 2 * ((int64_t)(i0 + c) * ldm + q0 + q))
                                                 : za;
        }
        __syncthreads();
#pragma unroll 2
        for (int q = 0; q < MQ; ++q) {
            const DFC a0 = Ys[2 * tp][q], a1 = Ys[2 * tp + 1][q];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const DFC mb = Ms[q][4 * tc + b];
                mac_conj(P[0][b], Q[0][b], a0, mb);
                mac_conj(P[1][b], Q[1][b], a1, mb);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int64_t p = p0 + 2 * tp + a;
        if (p >= n) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + 4 * tc + b;
            if (i >= r) continue;
            const DFPair v = conj_result(P[a][b], Q[a][b]);
            T[2 * (p * ldt + i)] = (double)v.hi.x + (double)v.lo.x;
            T[2 * (p * ldt + i) + 1] = (double)v.hi.y + (double)v.lo.y;
        }
    }
}

// Real: thread (tp, tc) owns rows p0 + 2 tp + {0,1}, columns i0 + 4 tc + {0..3}
// as two pairs of adjacent columns per row.
__global__ void __launch_bounds__(DF_THREADS)
    df_gemm_r_kernel(const double* Mt, int ldm, const double* Y, int64_t ldy, int64_t n, int k,
                     int r, double* T, int64_t ldt) {
    __shared__ float2 Ys[MP][MQ];
    __shared__ float2 Ms[MQ][MI];
    const int64_t p0 = (int64_t)blockIdx.x * MP;
    const int i0 = blockIdx.y * MI;
    const int tp = threadIdx.x / 8, tc = threadIdx.x % 8;
    DFPair S[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        zero(S[a][0]);
        zero(S[a][1]);
    }
    for (int q0 = 0; q0 < k; q0 += MQ) {
        for (int e = threadIdx.x; e < MP * MQ; e += DF_THREADS) {
            const int rr = e / MQ, c = e % MQ;
            const int64_t p = p0 + rr;
            Ys[rr][c] = (p < n && q0 + c < k) ? split_r(Y[p * ldy + q0 + c]) : make_float2(0.f, 0.f);
        }
        for (int e = threadIdx.x; e < MQ * MI; e += DF_THREADS) {
            const int q = e / MI, c = e % MI;
            Ms[q][c] = (q0 + q < k && i0 + c < r) ? split_r(Mt[(int64_t)(i0 + c) * ldm + q0 + q])
                                                 : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int q = 0; q < MQ; ++q) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float2 m0 = Ms[q][4 * tc + 2 * h], m1 = Ms[q][4 * tc + 2 * h + 1];
                DFPair mv;
                mv.hi = make_float2(m0.x, m1.x);
                mv.lo = make_float2(m0.y, m1.y);
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const float2 y = Ys[2 * tp + a][q];
                    df_mac(S[a][h], y.x, y.y, mv);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int64_t p = p0 + 2 * tp + a;
        if (p >= n) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const DFPair v = df_norm(S[a][h]);
            const int i = i0 + 4 * tc + 2 * h;
            if (i < r) T[p * ldt + i] = (double)v.hi.x + (double)v.lo.x;
            if (i + 1 < r) T[p * ldt + i + 1] = (double)v.hi.y + (double)v.lo.y;
        }
    }
}

}  // namespace

// C = conj(A^T-style) Gram of gemm_nh: C[i + j m] = sum_k A[k][i] conj(B[k][j]).
// `work` holds chunks * m * m float4 partials (see df_gram_work_bytes).
int df_gram_chunks(int m, int sms) {
    const int tiles = (m + GT - 1) / GT;
    return std::max(1, 8 * sms / (tiles * tiles));
}

size_t df_gram_work_bytes(int m, int sms) {
    return (size_t)df_gram_chunks(m, sms) * m * m * sizeof(float4);
}

void df_gram(bool cplx, const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n,
             int m, double* C, void* work, int sms, cudaStream_t s) {
    const int tiles = (m + GT - 1) / GT;
    const int chunks = df_gram_chunks(m, sms);
    int64_t rows = (n + chunks - 1) / chunks;
    rows = (rows + GR - 1) / GR * GR;
    const int used = (int)std::max<int64_t>(1, (n + rows - 1) / rows);
    dim3 grid(tiles * tiles, used);
    if (cplx)
        df_gram_c_kernel<<<grid, DF_THREADS, 0, s>>>(A, lda, B, ldb, n, m, rows, tiles,
                                                     (float4*)work);
    else
        df_gram_r_kernel<<<grid, DF_THREADS, 0, s>>>(A, lda, B, ldb, n, m, rows, tiles,
                                                     (float4*)work);
    const int64_t mm = (int64_t)m * m;
    const int g = (int)std::min<int64_t>((mm + 255) / 256, 4096);
    if (cplx)
        df_gram_reduce_kernel<true><<<g, 256, 0, s>>>((const float4*)work, used, m, C);
    else
        df_gram_reduce_kernel<false><<<g, 256, 0, s>>>((const float4*)work, used, m, C);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

// T (row-major n x r, ldt) = Y (row-major n x k, ldy) conj(M) with M column-major k x r (ldm).
void df_gemm(bool cplx, int r, int64_t n, int k, const double* Mt, int ldm, const double* Y,
             int64_t ldy, double* T, int64_t ldt, cudaStream_t s) {
    dim3 grid((unsigned)((n + MP - 1) / MP), (unsigned)((r + MI - 1) / MI));
    if (cplx)
        df_gemm_c_kernel<<<grid, DF_THREADS, 0, s>>>(Mt, ldm, Y, ldy, n, k, r, T, ldt);
    else
        df_gemm_r_kernel<<<grid, DF_THREADS, 0, s>>>(Mt, ldm, Y, ldy, n, k, r, T, ldt);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

}  // namespace chebfd
