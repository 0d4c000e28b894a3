// FP64-accurate tall Gram products C = A^H B (A, B: N x m blocks, FP64 real
// or complex, row-major) on the bf16 tensor cores, by an Ozaki-type split
// (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012)).  These are the Gram matrices
// of the orthonormalisation and Rayleigh-Ritz steps (Sec. 3.1 steps 6-7).
//
// A complex block is the real N x 2m block of its interleaved parts, so one
// real Gram G = A_r^T B_r (2m x 2m) gives every complex entry.  Each column
// of A_r (and of B_r) is scaled by a power of two 2^e (|entries| < 2^e) and
// written as a 56-bit fixed-point number, split into 8 balanced base-128
// digits d_1..d_8 (d_1 in [-128, 128], the others in [-64, 63]); every digit
// is an integer that bf16 holds exactly.  Then
//     G = 2^(e_a + e_b - 14) sum_{g} 2^(-7 (g - 2)) sum_{i + j = g} D_i^T E_j
// where D_i, E_j are the digit slices (N x 2m bf16).  Pairs with i + j <= 9
// (36 of 64) are kept; the dropped ones are below 2^-56 of the leading term.
//
// The slice products run as tcgen05.mma (kind::f16, bf16 in, FP32 out) into
// eight TMEM accumulators, one per group g = 2..9.  A product of two digits
// is at most 2^14 and a group has at most 7 x 2^12 per row in magnitude, so
// the groups g <= 6 stay exact integers in FP32 over 512 rows; every 512 rows
// they are read out, combined exactly into an int64 per output and cleared.
// The groups 7-9 (2^-35 and below) accumulate in FP32 over the whole range.
// Each CTA owns a 128 x 64 tile of G and a range of rows; a last kernel adds
// the ranges in a fixed order, applies the scales and forms the complex
// entries.  Digits are formed from the FP64 bit pattern with integer
// operations (FP64 arithmetic is slow on this GPU).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <mutex>
#include <vector>

#include "bulk_pipe.cuh"
#include "common.cuh"

namespace chebfd {

namespace {

constexpr int OZ_SLICES = 8;      // digits per entry
constexpr int OZ_GROUPS = 8;      // g = 2..9
constexpr int OZ_EXACT = 5;       // g = 2..6: exact, flushed every OZ_CHUNK rows
constexpr int OZ_BM = 128;        // tile rows (columns of A)
constexpr int OZ_BN = 64;         // tile columns (columns of B)
constexpr int OZ_BK = 64;         // rows per K-block (one 128-byte swizzle row of bf16)
constexpr int OZ_CHUNK = 512;     // rows between flushes of the exact groups
constexpr int OZ_A_STAGES = 5;    // ring of A slice tiles
constexpr int OZ_THREADS = 320;   // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int64_t OZ_MAX_RANGE = (int64_t)1 << 18;  // rows per CTA (int64 head-room)

constexpr int A_TILE_BYTES = OZ_BM * OZ_BK * 2;               // 16 KB
constexpr int B_STACK_BYTES = OZ_SLICES * OZ_BN * OZ_BK * 2;  // 64 KB

// ------------------------------------------------------------ tcgen05 / TMA

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, M = 128, bf16 inputs, FP32 accumulators.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrives (once) on bar when every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both
// K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(OZ_BM >> 4) << 24);
}

// Shared-memory descriptor of a K-major operand in the 128-byte swizzled
// layout the TMA writes (rows of 128 bytes, 8-row atoms of 1024 bytes).
__device__ __forceinline__ uint64_t umma_desc_sw128(const void* smem) {
    const uint64_t addr = smem_u32(smem);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;            // start address
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: 8 rows x 128 bytes
    d |= (uint64_t)1 << 46;                  // descriptor version
    d |= (uint64_t)2 << 61;                  // 128-byte swizzle
    return d;
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Zeros into 32 consecutive columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_zero32(uint32_t taddr) {
    const uint32_t z = 0;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
        "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(z)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// 3-D tiled TMA load of box {c0.., c1.., c2..} into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace

namespace {

// ------------------------------------------------------------ split into digits

// emax[c] = largest biased FP64 exponent field in column c of the N x cols
// block A (row-major, ldr doubles per row); atomically merged over blocks.
// Columns are handled 256 at a time by the threads of a block, up to 2048.
__global__ void oz_colexp_kernel(const double* __restrict__ A, int64_t n, int cols, int64_t ldr,
                                 int* __restrict__ emax) {
    int mx[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * per, r1 = min(n, r0 + per);
    for (int64_t r = r0; r < r1; ++r) {
        const unsigned long long* row = reinterpret_cast<const unsigned long long*>(A + r * ldr);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = threadIdx.x + 256 * q;
            if (c < cols) mx[q] = max(mx[q], (int)((__ldg(row + c) >> 52) & 0x7FF));
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int c = threadIdx.x + 256 * q;
        if (c < cols && mx[q] > 0) atomicMax(emax + c, mx[q]);
    }
}

// Exact float of a small integer (|v| < 2^22) without a conversion
// instruction: v added to the significand of 1.5 * 2^23, then 1.5 * 2^23
// subtracted (both exact).  A 64-bit integer-to-float conversion would run on
// the FP64 pipe, which is narrow on this part.
__device__ __forceinline__ float oz_small_float(int v) {
    return __fsub_rn(__int_as_float(0x4B400000 + v), 12582912.0f);
}

// The 8 balanced base-128 digits of x / 2^(E - 1022) as a 56-bit fixed-point
// number (E: the column's largest biased exponent field, so |x| < 2^(E-1022)).
__device__ __forceinline__ void oz_digits(double x, int E, float* d) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    unsigned long long mant = bits & ((1ull << 52) - 1);
    int e = ex;
    if (ex == 0) e = 1; else mant |= 1ull << 52;   // subnormal: no implicit bit
    // X = mant * 2^(e - E + 3) < 2^56, rounded to nearest when shifted right
    const int sh = e - E + 3;
    unsigned long long X;
    if (sh >= 0)
        X = mant << sh;
    else if (-sh >= 60)
        X = 0;
    else
        X = (mant + (1ull << (-sh - 1))) >> (-sh);
    long long V = (long long)X;
    if (bits >> 63) V = -V;
#pragma unroll
    for (int s = OZ_SLICES - 1; s >= 1; --s) {
        const int dv = (int)(((unsigned)V & 127u) ^ 64u) - 64;   // in [-64, 63]
        d[s] = oz_small_float(dv);
        V = (V - dv) >> 7;
    }
    d[0] = oz_small_float((int)V);                    // in [-128, 128]
}

// S[s][c][k] (bf16, k contiguous, kpad rows per column) = digit s of A[k][c];
// zero for n <= k < kpad.  A block takes 64 rows x 32 columns: lane = column
// (coalesced reads of a row), each thread forms the digits of two consecutive
// rows and keeps them as one 32-bit word per slice, so the transpose through
// shared memory (33 words per column: conflict-free) and the global writes
// (32 lanes x 4 bytes of one column) stay coalesced.
__global__ void __launch_bounds__(256) oz_split_kernel(const double* __restrict__ A, int64_t n,
                                                       int cols, int64_t ldr, const int* emax,
                                                       int64_t kpad, uint32_t* __restrict__ S) {
    __shared__ uint32_t t[OZ_SLICES][32][33];
    const int64_t k0 = (int64_t)blockIdx.x * 64;
    const int c0 = blockIdx.y * 32;
    const int tc = threadIdx.x % 32, tw = threadIdx.x / 32;
    const int c = c0 + tc;
    const int E = c < cols ? emax[c] : 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int kp = tw + 8 * p;           // row pair 0..31 of the tile
        const int64_t k = k0 + 2 * kp;
        float d0[OZ_SLICES], d1[OZ_SLICES];
        const double x0 = (c < cols && k < n) ? __ldg(A + k * ldr + c) : 0.0;
        const double x1 = (c < cols && k + 1 < n) ? __ldg(A + (k + 1) * ldr + c) : 0.0;
        oz_digits(x0, E, d0);
        oz_digits(x1, E, d1);
#pragma unroll
        for (int s = 0; s < OZ_SLICES; ++s) {
            const __nv_bfloat162 v = __floats2bfloat162_rn(d0[s], d1[s]);  // low half: row k
            t[s][tc][kp] = *reinterpret_cast<const uint32_t*>(&v);
        }
    }
    __syncthreads();
    // per (slice, column): 32 words (64 rows) written by the 32 lanes of a warp
    const size_t slice_stride = (size_t)cols * kpad / 2;   // in words
    for (int q = tw; q < OZ_SLICES * 32; q += 8) {
        const int s = q / 32, cc = q % 32;
        if (c0 + cc >= cols) continue;
        S[s * slice_stride + ((size_t)(c0 + cc) * kpad + k0) / 2 + tc] = t[s][cc][tc];
    }
}

}  // namespace

// Set when an Ozaki Gram kernel gave up a bounded wait; read by check_oz_errors().
__device__ unsigned int g_oz_error = 0;

namespace {

struct OzSmem {
    // 1024-byte aligned operand buffers first (the 128-byte swizzle atoms)
    unsigned char b[2][B_STACK_BYTES];        // 8 B slices of one K-block, double buffered
    unsigned char a[OZ_A_STAGES][A_TILE_BYTES];  // ring of single A slice tiles
    uint64_t a_full[OZ_A_STAGES], a_empty[OZ_A_STAGES];
    uint64_t b_full[2], b_empty[2];
    uint64_t chunk_done;                      // MMAs of a 512-row chunk completed
    uint64_t flushed;                         // epilogue has read and cleared the exact groups
    uint32_t tmem_base;
    uint32_t fail;                            // a bounded wait ran out somewhere in the CTA
};

__device__ __forceinline__ bool oz_wait(OzSmem& sm, uint64_t* bar, uint32_t parity) {
    if (*(volatile uint32_t*)&sm.fail) return false;
    if (mbar_wait(bar, parity)) return true;
    atomicExch(&sm.fail, 1u);
    atomicExch(&g_oz_error, kPipeErrTimeout);
    return false;
}

// Where a CTA's results go: without exponents, P[split][m][n] (ld = cols_b,
// split stride cols_a * cols_b) in units of one group-2 digit product; with
// the exponent fields ea[m], eb[n] (one split only), the finished values
// 2^(ea - 1022 + eb - 1022 - 14) x that at out[m * ld + n].
struct OzOut {
    double* P;
    int64_t ld;
    const int* ea;
    const int* eb;
    bool accumulate;  // add to P (the row chunks of a long Gram) instead of writing it
};

// v * 2^e: one exact multiplication when 2^e is a normal double, else ldexp.
__device__ __forceinline__ double oz_scale(double v, int e) {
    if (e >= -1022 && e <= 1023) return v * __longlong_as_double((long long)(e + 1023) << 52);
    return ldexp(v, e);
}

// The tiles of a Gram A^T A that reach the diagonal or lie above it (the
// rest are mirrored): row tile mi keeps the column tiles n0 >= m0 - (BN - 1),
// i.e. nj >= mi * BM / BN.  Linear index t -> (mi, nj).
__host__ __device__ inline int oz_upper_first(int mi) { return mi * (OZ_BM / OZ_BN); }
__host__ __device__ inline int oz_upper_tiles(int tm, int tn) {
    int c = 0;
    for (int mi = 0; mi < tm; ++mi) c += tn > oz_upper_first(mi) ? tn - oz_upper_first(mi) : 0;
    return c;
}

// One CTA: the 128 x 64 tile (m0, n0) of D = A_s B_s^T over the rows
// [k_begin, k_end) of the K dimension (k_begin a multiple of OZ_CHUNK), A_s
// and B_s the digit slices (rows x K, K contiguous).  upper_tn > 0: the grid's
// x index runs over the upper tiles of a tm x upper_tn Gram (A == B);
// upper_tn < 0: x is the column tile and y the row tile.
__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gram_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   int64_t rows_per_split, int64_t kpad, int64_t cols_a, int cols_b, OzOut o,
                   int upper_tn) {
    extern __shared__ unsigned char smem_raw[];
    OzSmem& sm = *reinterpret_cast<OzSmem*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int mi = blockIdx.x, nj = blockIdx.y;
    if (upper_tn < 0) {  // the block product: the column tiles of one row tile run together
        mi = blockIdx.y;
        nj = blockIdx.x;
    } else if (upper_tn > 0) {
        int t = blockIdx.x;
        mi = 0;
        // every row tile of a square Gram keeps at least one tile; at most 16 row tiles
        while (mi < 64 && t >= upper_tn - oz_upper_first(mi)) {
            t -= upper_tn - oz_upper_first(mi);
            ++mi;
        }
        nj = oz_upper_first(mi) + t;
    }
    const int64_t m0 = (int64_t)mi * OZ_BM;
    const int n0 = nj * OZ_BN, split = blockIdx.z;
    const int64_t k_begin = split * rows_per_split;
    const int64_t k_end = min(kpad, k_begin + rows_per_split);
    const int nkb = (int)((k_end - k_begin) / OZ_BK);          // kpad is a multiple of OZ_BK
    const int nchunks = (nkb + OZ_CHUNK / OZ_BK - 1) / (OZ_CHUNK / OZ_BK);

    if (threadIdx.x == 0) {
        for (int i = 0; i < OZ_A_STAGES; ++i) {
            mbar_init(&sm.a_full[i], 1);
            mbar_init(&sm.a_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sm.b_full[i], 1);
            mbar_init(&sm.b_empty[i], 1);
        }
        mbar_init(&sm.chunk_done, 1);
        mbar_init(&sm.flushed, 8);
        sm.fail = 0;
        mbar_init_fence();
    }
    if (warp == 1) {
        tmem_alloc(&sm.tmem_base, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;

    if (warp == 0) {
        // ---------------- TMA producer
        int issued_a = 0, issued_b = 0;
        if (lane == 0) {
            for (int kb = 0; kb < nkb; ++kb) {
                const int k = (int)(k_begin + (int64_t)kb * OZ_BK);
                const int bs = kb & 1;
                if (kb >= 2 && !oz_wait(sm, &sm.b_empty[bs], ((kb >> 1) - 1) & 1)) break;
                mbar_arrive_expect_tx(&sm.b_full[bs], B_STACK_BYTES);
                tma_load_3d(sm.b[bs], &tmB, k, n0, 0, &sm.b_full[bs]);
                ++issued_b;
                bool ok = true;
                for (int i = 0; i < OZ_SLICES && ok; ++i) {
                    const int q = kb * OZ_SLICES + i, as = q % OZ_A_STAGES;
                    if (q >= OZ_A_STAGES && !oz_wait(sm, &sm.a_empty[as], ((q / OZ_A_STAGES) - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&sm.a_full[as], A_TILE_BYTES);
                    tma_load_3d(sm.a[as], &tmA, k, (int)m0, i, &sm.a_full[as]);
                    ++issued_a;
                }
                if (!ok) break;
            }
            // every copy issued has landed before the CTA may end
            for (int q = max(0, issued_a - OZ_A_STAGES); q < issued_a; ++q)
                if (!mbar_wait(&sm.a_full[q % OZ_A_STAGES], (q / OZ_A_STAGES) & 1)) break;
            for (int kb = max(0, issued_b - 2); kb < issued_b; ++kb)
                if (!mbar_wait(&sm.b_full[kb & 1], (kb >> 1) & 1)) break;
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            bool ok = true;
            int committed_chunks = 0;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                const int c = kb / (OZ_CHUNK / OZ_BK);
                if (kb % (OZ_CHUNK / OZ_BK) == 0 && !oz_wait(sm, &sm.flushed, c & 1)) break;
                const int bs = kb & 1;
                if (!oz_wait(sm, &sm.b_full[bs], (kb >> 1) & 1)) break;
                tc_fence_after();
                for (int i = 0; i < OZ_SLICES; ++i) {
                    const int q = kb * OZ_SLICES + i, as = q % OZ_A_STAGES;
                    if (!oz_wait(sm, &sm.a_full[as], (q / OZ_A_STAGES) & 1)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t adesc = umma_desc_sw128(sm.a[as]);
                    // slice i+1 of A against slices j = 1 .. 8 - i of B: group i + j + 1,
                    // TMEM columns 64 (i + j - 1), at most 4 slices (256 columns) per MMA
                    for (int j0 = 1; j0 <= OZ_SLICES - i; j0 += 4) {
                        const int nj = min(4, OZ_SLICES - i - j0 + 1);
                        const uint64_t bdesc =
                            umma_desc_sw128(sm.b[bs] + (size_t)(j0 - 1) * OZ_BN * OZ_BK * 2);
                        const uint32_t d = tmem + (uint32_t)(OZ_BN * (i + j0 - 1));
                        const uint32_t idesc = umma_idesc_bf16(OZ_BN * nj);
#pragma unroll
                        for (int ks = 0; ks < OZ_BK / 16; ++ks)
                            // 16 rows of K = 32 bytes along the swizzled 128-byte row
                            umma_bf16(d, adesc + 2 * ks, bdesc + 2 * ks, idesc, 1u);
                    }
                    umma_commit(&sm.a_empty[as]);
                }
                if (!ok) break;
                umma_commit(&sm.b_empty[bs]);
                if (kb % (OZ_CHUNK / OZ_BK) == OZ_CHUNK / OZ_BK - 1 || kb == nkb - 1) {
                    umma_commit(&sm.chunk_done);
                    ++committed_chunks;
                }
            }
            // the MMAs in flight finish before TMEM is released: wait for the
            // last chunk commit (issued after every MMA)
            if (committed_chunks > 0)
                mbar_wait(&sm.chunk_done, (committed_chunks - 1) & 1);
        }
    } else {
        // ---------------- epilogue: warps 2..9
        const int quarter = warp % 4;              // TMEM lanes 32*quarter.. (hardware rule)
        const int half = (warp - 2) / 4;           // columns 32*half..32*half+31 of each group
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        auto col_addr = [&](int g) { return tmem + lane_base + (uint32_t)(OZ_BN * g + 32 * half); };
        for (int g = 0; g < OZ_GROUPS; ++g) tmem_zero32(col_addr(g));
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.flushed);
        long long T[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) T[j] = 0;
        bool ok = true;
        for (int c = 0; c < nchunks && ok; ++c) {
            bool got = true;
            if (lane == 0) got = oz_wait(sm, &sm.chunk_done, c & 1);
            ok = __shfl_sync(0xffffffffu, got, 0);
            if (!ok) break;
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < OZ_EXACT; ++g) {
                float v[32];
                tmem_ld32(col_addr(g), v);
                const int sh = 7 * (OZ_EXACT - 1 - g);
#pragma unroll
                for (int j = 0; j < 32; ++j) T[j] += (long long)__float2int_rn(v[j]) * (1ll << sh);
                tmem_zero32(col_addr(g));
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.flushed);
        }
        if (ok) {
            float t7[32], t8[32], t9[32];
            tmem_ld32(col_addr(OZ_EXACT), t7);
            tmem_ld32(col_addr(OZ_EXACT + 1), t8);
            tmem_ld32(col_addr(OZ_EXACT + 2), t9);
            const int64_t m = m0 + 32 * quarter + lane;
            if (m < cols_a) {
                double* out = o.P + ((size_t)split * cols_a + m) * o.ld;
                const int em = o.ea ? (o.ea[m] > 0 ? o.ea[m] - 1022 : 0) - 14 : 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int n = n0 + 32 * half + j;
                    if (n < cols_b) {
                        // the power-of-two weights folded into FMAs; groups 8 and 9
                        // (2^-7 and 2^-14 below group 7) combined in FP32: the FP64
                        // pipe, narrow on this part, does 6 operations per entry
                        const float t89 = fmaf(t9[j], 0x1p-7f, t8[j]);
                        double v = fma((double)t7[j], 0x1p-35,
                                       fma((double)t89, 0x1p-42, (double)T[j] * 0x1p-28));
                        if (o.ea) v = oz_scale(v, em + (o.eb[n] > 0 ? o.eb[n] - 1022 : 0));
                        out[n] = o.accumulate ? out[n] + v : v;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, 512);
}

// C (ma x mb, column-major, ldc) from the split partials: the fixed-order sum
// over splits, the column scales 2^(E_a - 1022) 2^(E_b - 1022) 2^-14, and for
// complex blocks the combination of the four real parts of each entry:
//     C[p + q ldc] = sum_i A[i,p] conj(B[i,q]).
// mirror: A == B and only the tiles on and above the diagonal were computed;
// a real entry (r, c) with r > c is read at (c, r).
__global__ void oz_finish_kernel(const double* __restrict__ P, int nsplit, int ca, int cb,
                                 int ma, int mb, bool cplx, const int* ea, const int* eb,
                                 double* __restrict__ C, int ldc, bool mirror) {
    const int total = ma * mb;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int p = t % ma, q = t / ma;
        auto g = [&](int r, int c) {
            if (mirror && r > c) {
                const int x = r;
                r = c;
                c = x;
            }
            double s = 0.0;
            for (int k = 0; k < nsplit; ++k) s += P[((size_t)k * ca + r) * cb + c];
            const int e = (ea[r] > 0 ? ea[r] - 1022 : 0) + (eb[c] > 0 ? eb[c] - 1022 : 0) - 14;
            return ldexp(s, e);
        };
        if (cplx) {
            const double re = g(2 * p, 2 * q) + g(2 * p + 1, 2 * q + 1);
            const double im = g(2 * p + 1, 2 * q) - g(2 * p, 2 * q + 1);
            C[2 * ((size_t)p + (size_t)q * ldc)] = re;
            C[2 * ((size_t)p + (size_t)q * ldc) + 1] = im;
        } else {
            C[(size_t)p + (size_t)q * ldc] = g(p, q);
        }
    }
}

}  // namespace

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    CHEBFD_REQUIRE(fn != nullptr, CHEBFD_ECUDA, "cuTensorMapEncodeTiled is not available");
    return fn;
}

// Tensor map of the digit slices S[8][cols][kpad] (bf16): box of OZ_BK rows x
// `rows` columns x `slices` slices, 128-byte swizzle (the layout the MMA
// descriptors expect), zero fill outside the block.
CUtensorMap slice_map(const __nv_bfloat16* S, int64_t kpad, int64_t cols, int rows, int slices) {
    CUtensorMap m;
    const cuuint64_t dim[3] = {(cuuint64_t)kpad, (cuuint64_t)cols, (cuuint64_t)OZ_SLICES};
    const cuuint64_t stride[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)cols * kpad * 2};
    const cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)rows, (cuuint32_t)slices};
    const cuuint32_t estride[3] = {1, 1, 1};
    const CUresult r = encode_tiled()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                                      const_cast<__nv_bfloat16*>(S), dim, stride, box, estride,
                                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CHEBFD_REQUIRE(r == CUDA_SUCCESS, CHEBFD_ECUDA,
                   "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return m;
}

struct OzBuf {
    void* p = nullptr;
    cudaStream_t s;
    OzBuf(size_t bytes, cudaStream_t st) : s(st) {
        if (bytes) CHEBFD_CHECK_CUDA(cudaMallocAsync(&p, bytes, st));
    }
    ~OzBuf() {
        if (p) cudaFreeAsync(p, s);
    }
    OzBuf(const OzBuf&) = delete;
    OzBuf& operator=(const OzBuf&) = delete;
};

// Column exponents (largest biased FP64 exponent field of each column) of one
// real N x cols block, over all N rows.
void oz_column_exponents(const double* A, int64_t n, int cols, int64_t ldr, int* emax, int sms,
                         cudaStream_t s) {
    CHEBFD_CHECK_CUDA(cudaMemsetAsync(emax, 0, (size_t)cols * sizeof(int), s));
    const int g = (int)std::min<int64_t>((int64_t)sms * 8, std::max<int64_t>(1, n / 64));
    oz_colexp_kernel<<<g, 256, 0, s>>>(A, n, cols, ldr, emax);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

// Digit slices S[8][cols][kpad] of the rows [0, n) of a real block whose
// column exponents are emax (rows n..kpad-1 zero).
void oz_split_rows(const double* A, int64_t n, int cols, int64_t ldr, int64_t kpad,
                   const int* emax, __nv_bfloat16* S, cudaStream_t s) {
    const dim3 grid((unsigned)(kpad / 64), (unsigned)((cols + 31) / 32));
    oz_split_kernel<<<grid, 256, 0, s>>>(A, n, cols, ldr, emax, kpad,
                                         reinterpret_cast<uint32_t*>(S));
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------ block products

// e[r] = largest biased exponent field of row r (kreal entries, ldr doubles
// apart between rows): one warp per row.
__global__ void oz_rowexp_kernel(const double* __restrict__ A, int64_t rows, int kreal,
                                 int64_t ldr, int* __restrict__ e) {
    const int lane = threadIdx.x % 32;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t r = w0; r < rows; r += nw) {
        const unsigned long long* row = reinterpret_cast<const unsigned long long*>(A + r * ldr);
        unsigned mx = 0;
        for (int k = lane; k < kreal; k += 32) mx = max(mx, (unsigned)((__ldg(row + k) >> 52) & 0x7FF));
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) e[r] = (int)mx;
    }
}

// S[s][r][k] (bf16, kpad per row) = digit s of A[r][k] with the row's scale;
// zero for kreal <= k < kpad.  One thread per pair of entries (one 32-bit
// word per slice): reads and writes run along the row.
__global__ void oz_rowsplit_kernel(const double* __restrict__ A, int64_t rows, int kreal,
                                   int64_t ldr, const int* __restrict__ e, int64_t kpad,
                                   uint32_t* __restrict__ S) {
    const int64_t words = kpad / 2, total = rows * words;
    const size_t slice_stride = (size_t)rows * words;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / words, j = t - r * words;
        const int E = e[r];
        const int k = (int)(2 * j);
        const double x0 = k < kreal ? __ldg(A + r * ldr + k) : 0.0;
        const double x1 = k + 1 < kreal ? __ldg(A + r * ldr + k + 1) : 0.0;
        float d0[OZ_SLICES], d1[OZ_SLICES];
        oz_digits(x0, E, d0);
        oz_digits(x1, E, d1);
#pragma unroll
        for (int s = 0; s < OZ_SLICES; ++s) {
            const __nv_bfloat162 v = __floats2bfloat162_rn(d0[s], d1[s]);
            S[s * slice_stride + t] = *reinterpret_cast<const uint32_t*>(&v);
        }
    }
}

// Rows of the right operand for T = Y W, W = conj(M) (conj) or M, M a k x r
// column-major matrix (ldm): real B[i][q] = W(q, i); complex, on the
// interleaved real views, B[2i][2q] = Re W, B[2i][2q+1] = -Im W,
// B[2i+1][2q] = Im W, B[2i+1][2q+1] = Re W (row-major, kreal per row).
__global__ void oz_build_b_kernel(const double* __restrict__ M, int ldm, int k, int r, bool cplx,
                                  bool conj, double* __restrict__ Bh) {
    const int total = k * r;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int q = t % k, i = t / k;
        if (!cplx) {
            Bh[(size_t)i * k + q] = M[q + (size_t)i * ldm];
            continue;
        }
        const double re = M[2 * (q + (size_t)i * ldm)];
        const double im = conj ? -M[2 * (q + (size_t)i * ldm) + 1] : M[2 * (q + (size_t)i * ldm) + 1];
        const size_t kr = 2 * (size_t)k;
        Bh[(2 * (size_t)i) * kr + 2 * q] = re;
        Bh[(2 * (size_t)i) * kr + 2 * q + 1] = -im;
        Bh[(2 * (size_t)i + 1) * kr + 2 * q] = im;
        Bh[(2 * (size_t)i + 1) * kr + 2 * q + 1] = re;
    }
}

void oz_prepare_rows(const double* A, int64_t rows, int kreal, int64_t ldr, int64_t kpad, int* e,
                     __nv_bfloat16* S, int sms, cudaStream_t s) {
    const int g = (int)std::min<int64_t>((int64_t)sms * 16, std::max<int64_t>(1, (rows + 7) / 8));
    oz_rowexp_kernel<<<g, 256, 0, s>>>(A, rows, kreal, ldr, e);
    const int64_t work = rows * (kpad / 2);
    const int g2 = (int)std::min<int64_t>((int64_t)sms * 32, std::max<int64_t>(1, (work + 255) / 256));
    oz_rowsplit_kernel<<<g2, 256, 0, s>>>(A, rows, kreal, ldr, e, kpad,
                                          reinterpret_cast<uint32_t*>(S));
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

}  // namespace

size_t oz_gram_smem_bytes() { return sizeof(OzSmem) + 1024; }

// Bytes of digit slices the tall products keep at a time: longer blocks are
// processed in row chunks (a Gram keeps the column exponents of the whole
// block, and split j of every chunk adds its partial into the same FP64
// slot, chunk after chunk; the block product's rows are independent).
constexpr int64_t OZ_WORKSPACE_BYTES = 2LL << 30;

// C (ma x mb, column-major, ld ma) with C[p + q ma] = sum_i A[i,p] conj(B[i,q])
// for row-major blocks A (N x ma, lda) and B (N x mb, ldb), FP64 real or
// complex (interleaved); B == A (same shape) is recognised: split once, and
// only the tiles on and above the diagonal computed.  Asynchronous on s;
// workspace from the stream-ordered allocator.
void oz_gram_rect(bool cplx, const double* A, int64_t lda, int ma, const double* B, int64_t ldb,
                  int mb, int64_t n, double* C, int sms, cudaStream_t s) {
    cache_stream_workspace();
    const int ca = cplx ? 2 * ma : ma, cb = cplx ? 2 * mb : mb;
    const int64_t ldra = cplx ? 2 * lda : lda, ldrb = cplx ? 2 * ldb : ldb;
    CHEBFD_REQUIRE(ca >= 1 && cb >= 1 && ca <= 2048 && cb <= 2048, CHEBFD_EINVAL,
                   "Ozaki Gram: between 1 and 2048 real columns per operand");
    CHEBFD_REQUIRE(n >= 1, CHEBFD_EINVAL, "Ozaki Gram: empty block");
    const bool same = A == B && lda == ldb && ma == mb;
    OzBuf ea((size_t)ca * sizeof(int), s), eb(same ? 0 : (size_t)cb * sizeof(int), s);
    oz_column_exponents(A, n, ca, ldra, (int*)ea.p, sms, s);
    if (!same) oz_column_exponents(B, n, cb, ldrb, (int*)eb.p, sms, s);
    const int* eB = same ? (const int*)ea.p : (const int*)eb.p;
    // rows per chunk: a multiple of OZ_CHUNK within the workspace
    const int64_t slice_bytes_per_row = (int64_t)OZ_SLICES * (ca + (same ? 0 : cb)) * 2;
    int64_t rows_c = std::max<int64_t>(
        OZ_CHUNK, OZ_WORKSPACE_BYTES / slice_bytes_per_row / OZ_CHUNK * OZ_CHUNK);
    if (rows_c >= n) rows_c = n;
    const int64_t nchunk = (n + rows_c - 1) / rows_c;
    const int64_t kpad_max = (rows_c + OZ_BK - 1) / OZ_BK * OZ_BK;
    OzBuf sa((size_t)OZ_SLICES * ca * kpad_max * sizeof(__nv_bfloat16), s);
    OzBuf sb(same ? 0 : (size_t)OZ_SLICES * cb * kpad_max * sizeof(__nv_bfloat16), s);
    const __nv_bfloat16* SB = same ? (const __nv_bfloat16*)sa.p : (const __nv_bfloat16*)sb.p;
    // K-splits of each chunk: rows per CTA a multiple of OZ_CHUNK, at most
    // OZ_MAX_RANGE, enough splits that the tiles x splits fill the SMs
    const int tm = (ca + OZ_BM - 1) / OZ_BM, tn = (cb + OZ_BN - 1) / OZ_BN;
    const int tiles = same ? oz_upper_tiles(tm, tn) : tm * tn;
    std::vector<int64_t> nsplit(nchunk), range(nchunk);
    int64_t max_splits = 0;
    for (int64_t c = 0; c < nchunk; ++c) {
        const int64_t rows = std::min(rows_c, n - c * rows_c);
        const int64_t kpad = (rows + OZ_BK - 1) / OZ_BK * OZ_BK;
        const int64_t chunks = (kpad + OZ_CHUNK - 1) / OZ_CHUNK;
        int64_t ns = std::max<int64_t>(1, std::min<int64_t>(chunks, sms / std::max(1, tiles)));
        int64_t rg = (chunks + ns - 1) / ns * OZ_CHUNK;
        if (rg > OZ_MAX_RANGE) rg = OZ_MAX_RANGE;
        nsplit[c] = (kpad + rg - 1) / rg;
        range[c] = rg;
        max_splits = std::max(max_splits, nsplit[c]);
    }
    // split j of every chunk adds into P[j]; the chunks run in order on s
    OzBuf P((size_t)max_splits * ca * cb * sizeof(double), s);
    CHEBFD_CHECK_CUDA(
        cudaMemsetAsync(P.p, 0, (size_t)max_splits * ca * cb * sizeof(double), s));
    const size_t smem = oz_gram_smem_bytes();
    ensure_dynamic_smem(reinterpret_cast<const void*>(oz_gram_kernel), smem);
    for (int64_t c = 0; c < nchunk; ++c) {
        const int64_t r0 = c * rows_c, rows = std::min(rows_c, n - r0);
        const int64_t kpad = (rows + OZ_BK - 1) / OZ_BK * OZ_BK;
        oz_split_rows(A + r0 * ldra, rows, ca, ldra, kpad, (const int*)ea.p,
                      (__nv_bfloat16*)sa.p, s);
        if (!same)
            oz_split_rows(B + r0 * ldrb, rows, cb, ldrb, kpad, eB, (__nv_bfloat16*)sb.p, s);
        const CUtensorMap tmA = slice_map((const __nv_bfloat16*)sa.p, kpad, ca, OZ_BM, 1);
        const CUtensorMap tmB = slice_map(SB, kpad, cb, OZ_BN, OZ_SLICES);
        const dim3 grid = same ? dim3((unsigned)tiles, 1u, (unsigned)nsplit[c])
                               : dim3((unsigned)tm, (unsigned)tn, (unsigned)nsplit[c]);
        const OzOut o{(double*)P.p, cb, nullptr, nullptr, true};
        oz_gram_kernel<<<grid, OZ_THREADS, smem, s>>>(tmA, tmB, range[c], kpad, ca, cb, o,
                                                      same ? tn : 0);
        CHEBFD_CHECK_CUDA(cudaGetLastError());
    }
    const int total = ma * mb;
    oz_finish_kernel<<<std::min(4096, (total + 255) / 256), 256, 0, s>>>(
        (const double*)P.p, (int)max_splits, ca, cb, ma, mb, cplx, (const int*)ea.p, eB, C, ma,
        same);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

// The square case: C (m x m, ld m) = sum_i A[i,p] conj(B[i,q]).
void oz_gram(bool cplx, const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n,
             int m, double* C, int sms, cudaStream_t s) {
    oz_gram_rect(cplx, A, lda, m, B, ldb, m, n, C, sms, s);
}

// T[p][i] = sum_q Y[p][q] W(q, i), W = conj(M) if conj else M, for a row-major
// N x k block Y (ldy) and a k x r column-major M (ldm), FP64 real or complex,
// into T (N x r, ldt; must not overlap Y), at FP64 accuracy on the bf16 tensor
// cores: the digit slices of Y (per-row scales) and of the rows of W^T (per
// output column), K = k real or 2k (complex) in chunks of 512, no row split.
// Asynchronous on s; workspace from the stream-ordered allocator.
void oz_gemm(bool cplx, int r, int64_t n, int k, const double* M, int ldm, const double* Y,
             int64_t ldy, double* T, int64_t ldt, int sms, cudaStream_t s, bool conj) {
    CHEBFD_REQUIRE(n >= 1 && k >= 1 && r >= 1, CHEBFD_EINVAL, "Ozaki block product: empty operand");
    CHEBFD_REQUIRE(n < (1LL << 31), CHEBFD_EINVAL, "Ozaki block product: N must be < 2^31");
    cache_stream_workspace();
    const int kreal = cplx ? 2 * k : k, rows_b = cplx ? 2 * r : r;
    const int64_t kpad = (kreal + OZ_BK - 1) / OZ_BK * OZ_BK;
    const int64_t range = (kpad + OZ_CHUNK - 1) / OZ_CHUNK * OZ_CHUNK;
    CHEBFD_REQUIRE(range <= OZ_MAX_RANGE, CHEBFD_EINVAL, "Ozaki block product: k too large");
    const int64_t ldry = cplx ? 2 * ldy : ldy, ldrt = cplx ? 2 * ldt : ldt;
    // rows of Y per chunk: a multiple of OZ_BM within the workspace
    int64_t rows_c = std::max<int64_t>(
        OZ_BM, OZ_WORKSPACE_BYTES / ((int64_t)OZ_SLICES * kpad * 2) / OZ_BM * OZ_BM);
    if (rows_c >= n) rows_c = n;
    OzBuf ea((size_t)rows_c * sizeof(int), s), eb((size_t)rows_b * sizeof(int), s);
    OzBuf sa((size_t)OZ_SLICES * rows_c * kpad * sizeof(__nv_bfloat16), s);
    OzBuf bh((size_t)rows_b * kreal * sizeof(double), s);
    OzBuf sb((size_t)OZ_SLICES * rows_b * kpad * sizeof(__nv_bfloat16), s);
    oz_build_b_kernel<<<std::min(1024, (k * r + 255) / 256), 256, 0, s>>>(M, ldm, k, r, cplx, conj,
                                                                          (double*)bh.p);
    oz_prepare_rows((const double*)bh.p, rows_b, kreal, kreal, kpad, (int*)eb.p,
                    (__nv_bfloat16*)sb.p, sms, s);
    const CUtensorMap tmB = slice_map((const __nv_bfloat16*)sb.p, kpad, rows_b, OZ_BN, OZ_SLICES);
    const size_t smem = oz_gram_smem_bytes();
    ensure_dynamic_smem(reinterpret_cast<const void*>(oz_gram_kernel), smem);
    for (int64_t r0 = 0; r0 < n; r0 += rows_c) {
        const int64_t rows = std::min(rows_c, n - r0);
        oz_prepare_rows(Y + r0 * ldry, rows, kreal, ldry, kpad, (int*)ea.p, (__nv_bfloat16*)sa.p,
                        sms, s);
        const CUtensorMap tmA = slice_map((const __nv_bfloat16*)sa.p, kpad, rows, OZ_BM, 1);
        // x: the column tiles of one row tile, consecutive, so they share its
        // A slices in L2
        const unsigned tm = (unsigned)((rows + OZ_BM - 1) / OZ_BM);
        const unsigned tn = (unsigned)((rows_b + OZ_BN - 1) / OZ_BN);
        const OzOut o{T + r0 * ldrt, ldrt, (const int*)ea.p, (const int*)eb.p, false};
        oz_gram_kernel<<<dim3(tn, tm, 1), OZ_THREADS, smem, s>>>(tmA, tmB, range, kpad, rows,
                                                                 rows_b, o, -1);
        CHEBFD_CHECK_CUDA(cudaGetLastError());
    }
}

// Up to 4 GiB of the stream-ordered pool stays cached across the stream
// synchronisations of the solve (the default keeps none, so every call would
// map its workspace again).  Once per device, for this process's default pool.
void cache_stream_workspace() {
    static std::once_flag once[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::call_once(once[dev], [dev] {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
        uint64_t keep = 4ull << 30;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    });
}

// CHEBFD_ETIMEOUT if an Ozaki Gram kernel gave up a bounded wait since the
// last check (the flag is then cleared).  Synchronizes the stream.
void check_oz_errors(cudaStream_t s) {
    unsigned int h = 0;
    CHEBFD_CHECK_CUDA(cudaMemcpyFromSymbolAsync(&h, g_oz_error, sizeof(h), 0,
                                                cudaMemcpyDeviceToHost, s));
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
    if (h != 0) {
        const unsigned int zero = 0;
        CHEBFD_CHECK_CUDA(cudaMemcpyToSymbolAsync(g_oz_error, &zero, sizeof(zero), 0,
                                                  cudaMemcpyHostToDevice, s));
        CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
        CHEBFD_REQUIRE(false, CHEBFD_ETIMEOUT,
                       "the tensor-core Gram gave up waiting for its pipeline stages");
    }
}

}  // namespace chebfd
