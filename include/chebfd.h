/*
 * chebfd.h - C ABI of the GB300 (sm_103a) Chebyshev filter diagonalization
 * library libchebfd.so.
 *
 * Method: Pieper, Kreutzer, Alvermann, Galgon, Fehske, Hager, Lang, Wellein,
 * "High-performance implementation of Chebyshev filter diagonalization for
 * interior eigenvalue computations" (arXiv 1510.04895).  Problem statement
 * (Sec. 2): given a sparse Hermitian H, find the eigenpairs (lambda, v) with
 * lambda in [lam_lo, lam_hi] and ||H v - lambda v|| <= eps.
 *
 * Conventions shared by every entry point
 *  - Every function returns chebfd_status; CHEBFD_OK (0) is success.  No C++
 *    exception crosses the ABI.  chebfd_last_error() returns a thread-local
 *    message describing the last failure of the calling thread.
 *  - Ownership: the caller owns every pointer it passes in and keeps it alive
 *    for the duration of the call (and, for device buffers used by work queued
 *    on `stream`, until that work has completed).  The library owns the opaque
 *    handles (chebfd_matrix, chebfd_result) and frees them in *_destroy.
 *  - Block vectors are N x nb, ROW-MAJOR (interleaved: row i, vector k at
 *    X[i*ld + k], Sec. 4 "storage of block vectors in row major order"),
 *    resident in device memory, with ld >= nb in elements.  The base pointer,
 *    ld*element_size and nb*element_size must be multiples of 16 bytes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is queued on it; a call returns without waiting
 *    unless its comment says that it synchronizes.
 *  - Scalars: chebfd_dtype names the element type of vectors and matrix
 *    values.  A complex H (insulator) takes C128/C64 vectors, a real H
 *    (graphene, diagonal) takes R64/R32 vectors.
 *  - Workspace comes from the CUDA stream-ordered allocator (the device's
 *    default memory pool).  The first call that uses the tensor-core dense
 *    products sets that pool's release threshold to 4 GiB for the rest of
 *    the process, so up to 4 GiB of freed workspace stays reserved across
 *    stream synchronisations instead of being mapped again on every call;
 *    a process-local setting of the pool, not of the GPU.
 */
#ifndef CHEBFD_H
#define CHEBFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CHEBFD_ABI_VERSION 3

typedef enum chebfd_status {
    CHEBFD_OK = 0,
    CHEBFD_EINVAL = 1,       /* bad argument (null pointer, size, alignment, dtype) */
    CHEBFD_ENOMEM = 2,       /* device or host allocation failed */
    CHEBFD_ECUDA = 3,        /* a CUDA runtime / cuBLAS / cuSOLVER call failed */
    CHEBFD_ENUMERIC = 4,     /* NaN, or the recurrence diverged: spec(H) not inside [a,b] */
    CHEBFD_ENOCONV = 5,      /* iteration limit reached before convergence */
    CHEBFD_ETIMEOUT = 6,     /* a bounded device-side wait gave up */
    CHEBFD_EUNSUPPORTED = 7  /* valid request the library does not implement */
} chebfd_status;

typedef enum chebfd_dtype {
    CHEBFD_R64 = 0,   /* double */
    CHEBFD_C128 = 1,  /* complex double, (re, im) interleaved */
    CHEBFD_R32 = 2,   /* float */
    CHEBFD_C64 = 3    /* complex float, (re, im) interleaved */
} chebfd_dtype;

/* Damping kernels g_n of Tab. Kernel (Sec. 2.1); NONE is g_n = 1 (Sec. 2.3). */
typedef enum chebfd_kernel {
    CHEBFD_KERNEL_NONE = 0,
    CHEBFD_KERNEL_FEJER = 1,
    CHEBFD_KERNEL_JACKSON = 2,
    CHEBFD_KERNEL_LANCZOS = 3
} chebfd_kernel;

typedef enum chebfd_lattice_kind {
    CHEBFD_LATTICE_TOPI = 0,      /* 3D topological insulator, periodic (Sec. 5.1 pattern) */
    CHEBFD_LATTICE_GRAPHENE = 1,  /* 2D honeycomb lattice with onsite disorder (Sec. 5.4) */
    CHEBFD_LATTICE_TOPI_SLAB = 2  /* the paper's Eq. Ham: insulator slab, open in z */
} chebfd_lattice_kind;

/* Description of a generated lattice Hamiltonian.
 *  TOPI: Lx*Ly*Lz sites, 4 orbitals, row = 4*(x + Lx*(y + Ly*z)) + orbital,
 *    onsite (m + V_s) Gamma1, hopping T_j = -(t/2)(Gamma1 - i Gamma_{j+1}) from
 *    site s to s+e_j plus Hermitian conjugate, periodic; 13 entries per row
 *    (N_nzr = 13, Sec. 4).  Gamma1 = sz(x)s0, Gamma2 = sx(x)sx,
 *    Gamma3 = sx(x)sy, Gamma4 = sx(x)sz.
 *  TOPI_SLAB: Eq. Ham of Sec. 5.1: the same hopping, onsite V_s Gamma0 +
 *    m Gamma1 (Gamma0 = identity; the paper has m = 2), periodic in x and y and
 *    open in z (a slab of Lz layers): 11 entries in the rows of the two
 *    surface layers, 13 elsewhere.  Onsite values V_s + m and V_s - m.
 *  GRAPHENE: Lx*Ly cells, row = 2*(i + Lx*j) + sublattice, hopping -t to the
 *    three nearest neighbours, onsite V; 4 entries per row (N_nzr = 4, Sec. 4).
 *    Lz and m are ignored.
 *  Disorder V = W*(u - 1/2), u = top 53 bits of the SplitMix64 word number
 *  `index` (site for TOPI, row for GRAPHENE) of the generator started at state
 *  seed*256 + 0, times 2^-53.  Columns ascend within a row; coinciding entries
 *  (edges of length <= 2) are summed in the order onsite, +x, -x, +y, -y, +z, -z.
 *  Values are generated in FP64 (C128 for TOPI, R64 for GRAPHENE). */
typedef struct chebfd_lattice_desc {
    int32_t kind;        /* chebfd_lattice_kind */
    int32_t Lx, Ly, Lz;  /* lattice edges, each >= 1 */
    double t, m, W;      /* hopping, mass (TOPI), disorder strength */
    uint64_t seed;       /* disorder seed, < 2^56 */
    int32_t sell_C;      /* SELL chunk height C in {1,2,4,8,16,32} */
    int32_t sell_sigma;  /* SELL sorting window sigma >= 1 */
    int32_t also_single; /* nonzero: also keep a C64 / R32 copy of the values */
    int32_t reserved;
} chebfd_lattice_desc;

typedef struct chebfd_matrix chebfd_matrix;

typedef struct chebfd_matrix_info {
    int64_t n;            /* dimension D */
    int64_t nnz;          /* stored entries without SELL padding */
    int64_t nnz_padded;   /* SELL slots = chunk_ptr[nchunks] */
    int64_t nchunks;      /* ceil(n / C) */
    int32_t C, sigma;     /* SELL-C-sigma parameters */
    int32_t max_row_len;
    int32_t is_complex;   /* values C128 (and C64) if nonzero, else R64 (and R32) */
    int32_t has_single;   /* a single-precision copy of the values exists */
    int32_t blocked_width; /* block columns per 4-row block of the blocked copy, 0 if none */
} chebfd_matrix_info;

/* ------------------------------------------------------------------ basics */

int chebfd_abi_version(void);
const char* chebfd_last_error(void);
const char* chebfd_status_string(chebfd_status s);

/* ----------------------------------------------------------- matrix (D1) */

/* Build the device SELL-C-sigma matrix (Sec. 4: SELL-32-1 for one vector,
 * SELL-1-1 for blocks; format of Kreutzer et al. 2014) from a HOST CSR.
 * rowptr[n+1] (int64, rowptr[0] = 0), col[rowptr[n]] (int32, 0 <= col < n),
 * val[rowptr[n]] of dtype val_dtype in {R64, C128}; the matrix must be
 * Hermitian (not checked).  Rows are stably sorted by decreasing length inside
 * windows of sell_sigma rows, cut into chunks of sell_C rows, padded to the
 * chunk's longest row with (column = own row, value 0) and stored column-major
 * within each chunk.  also_single != 0 also stores R32/C64 values (round to
 * nearest).  Synchronizes `stream`.  EINVAL on bad sizes, ENOMEM, ECUDA. */
chebfd_status chebfd_matrix_create_csr(int64_t n, const int64_t* rowptr, const int32_t* col,
                                       const void* val, chebfd_dtype val_dtype, int sell_C,
                                       int sell_sigma, int also_single, void* stream,
                                       chebfd_matrix** out);

/* Generate a lattice Hamiltonian (see chebfd_lattice_desc) directly on the
 * device and store it as SELL-C-sigma.  Synchronizes `stream`. */
chebfd_status chebfd_matrix_create_lattice(const chebfd_lattice_desc* desc, void* stream,
                                           chebfd_matrix** out);

chebfd_status chebfd_matrix_get_info(const chebfd_matrix* H, chebfd_matrix_info* out);

/* Copy the SELL arrays to HOST buffers sized from chebfd_matrix_get_info:
 * chunk_ptr[nchunks+1] int64, chunk_len[nchunks] int32, col[nnz_padded] int32,
 * val[nnz_padded] FP64 values (R64 or C128), perm[n] int64 (original row of
 * sorted row r).  Any pointer may be NULL to skip that array.  Synchronous. */
chebfd_status chebfd_matrix_export_sell(const chebfd_matrix* H, int64_t* chunk_ptr,
                                        int32_t* chunk_len, int32_t* col, void* val,
                                        int64_t* perm);

/* Blocked copy.  A complex matrix built with also_single, sell_sigma = 1 and
 * n divisible by 4 whose blocks of 4 consecutive rows (the orbitals of one
 * lattice site, Sec. 4's topological insulator) each couple to at most 7
 * blocks of 4 columns and hold on average at least 28 stored entries (so the
 * dense blocks store at most 4x the entries) also gets a blocked-ELL copy:
 * per row block, 7 block columns (own block first) with dense 4x4 complex64
 * blocks (zeros stored).
 * The complex64 Chebyshev step (chebfd_chebyshev_step and the loop of
 * chebfd_filter_block) then reads that copy and computes the 4 rows of a
 * block together, gathering each neighbour row of u once per block instead
 * of once per row; results agree with the SELL kernel to FP32 rounding.  It
 * costs 7 * 16 * 8 = 896 bytes per 4 rows of device memory.  The copy is not
 * built when the environment variable CHEBFD_BLOCKED is "0" at creation.
 * chebfd_matrix_set_blocked(H, 0) makes the kernels use the SELL arrays only;
 * (H, 1) uses the copy again (EUNSUPPORTED if there is none).  Not thread-safe
 * against kernels of H in flight on other host threads. */
chebfd_status chebfd_matrix_set_blocked(chebfd_matrix* H, int enable);

/* Matrix-free step (the paper's "constructed on-the-fly" matrices, Sec. 1).
 * For an insulator lattice (TOPI or TOPI_SLAB) built with also_single and
 * sell_sigma = 1, chebfd_matrix_set_matrix_free(H, 1) makes the complex64
 * Chebyshev step (chebfd_chebyshev_step and the loop of chebfd_filter_block)
 * and the double-float step (the loop of chebfd_filter_block_df and of the
 * MIXED_DF solve's sweeps) rebuild H's entries in registers from the lattice
 * description (hopping t/2 blocks, onsite m +- V_s with V_s regenerated from
 * the SplitMix64 disorder stream) instead of reading any stored matrix: the
 * step then moves only the vectors.  The other operations keep using the
 * stored arrays.  Results agree with the stored-matrix kernels to FP32
 * (complex64) or double-float rounding.
 * (H, 0) returns to the stored matrix.  EUNSUPPORTED for other matrices.
 * (H, 2): as (H, 1), and the complex64 filter (chebfd_filter_block) runs
 * the steps two at a time (temporal blocking): 16-column panels, 8 x 8 x-y
 * tiles with a one-site halo and z-segments of Z planes (Z divides Lz; Lx,
 * Ly multiples of 8), T_{n+1} of the tile and its halo kept in a ring of
 * three planes in shared memory, so a pair of steps moves the vectors 6
 * times instead of 10; results equal the single steps bit for bit.  On
 * GB300 this is slower than the single step (latency-bound at 8 warps per
 * SM), so it is off by default.  EINVAL for other modes. */
chebfd_status chebfd_matrix_set_matrix_free(chebfd_matrix* H, int enable);

chebfd_status chebfd_matrix_destroy(chebfd_matrix* H);

/* ------------------------------------------------------------ kernels (K1) */

/* Y = (alpha H + beta) X for a device block X (N x nb, ld), Y of the same
 * shape (Y != X).  vdt selects the vector type and the matching value copy.
 * Wider blocks than one kernel row group (C128/C64: 64, R64/R32: 128 columns)
 * are processed as column panels.  Asynchronous on `stream`. */
chebfd_status chebfd_spmv(const chebfd_matrix* H, double alpha, double beta, const void* X,
                          void* Y, int64_t ld, int nb, chebfd_dtype vdt, void* stream);

/* ------------------------------------------------ bounds and scaling (A1-A2) */

/* Spectral interval [a, b] from `lanczos_steps` Lanczos steps (Sec. 3.1 step
 * 1: 20-30 steps), FP64, full reorthogonalisation, start vector of SplitMix64
 * stream 4 (entries 2u-1).  a = theta_min - rho_min, b = theta_max + rho_max
 * (rho = Ritz residual bound |beta_m s_m,i|), widened by 1% of b-a on each side
 * and clamped to the Gershgorin interval.  alpha = 2/(b-a), beta = (a+b)/(a-b)
 * (Eq. W1).  All outputs are HOST scalars; any may be NULL.  Synchronizes. */
chebfd_status chebfd_scale_bounds(const chebfd_matrix* H, int lanczos_steps, uint64_t seed,
                                  double* a, double* b, double* alpha, double* beta,
                                  void* stream);

/* ------------------------------------------------------- coefficients (A3-A4) */

/* gc[n] = g_n c_n, n = 0..Np, into a HOST array of Np+1 doubles: c_n are the
 * Chebyshev coefficients of the rectangular window [lam_lo, lam_hi] inside
 * [a, b] (Sec. 2.1, taken with the sign that makes p ~ +1 in the window:
 * c_0 = (th_lo - th_hi)/pi, c_n = 2/(pi n)(sin n th_lo - sin n th_hi),
 * th = arccos(alpha lam + beta) clamped), g_n the kernel factors of Tab. Kernel
 * (mu is the Lanczos exponent, ignored otherwise).  Pure host math. */
chebfd_status chebfd_window_coeffs(double a, double b, double lam_lo, double lam_hi, int Np,
                                   chebfd_kernel kernel, double mu, double* gc);

/* ---------------------------------------------------- filter (A5, K2, K4) */

/* Replace the device block X (N x nb, row-major, ld) by p[H] X =
 * sum_{n=0}^{Np} gc[n] T_n(alpha H + beta) X, following Fig. ChebFD: two start
 * steps, then for n = 3..Np one fused kernel per step computing
 * w <- 2(alpha H + beta) u - w and X <- X + gc[n] w in a single pass over the
 * matrix and the vectors.  Np >= 2; gc is a HOST array of Np+1 doubles.
 * If `moments` (DEVICE, 2*Np x nb doubles, row n = moment n) is non-NULL the
 * same passes also produce the Chebyshev moments mu_n[k] = <x_k, T_n(A) x_k>
 * of Sec. 4 (via mu_2n = 2<u_n,u_n> - mu_0, mu_2n+1 = 2<u_n+1,u_n> - mu_1),
 * and the call synchronizes `stream` and returns ENUMERIC if a moment is NaN or
 * |mu_2n| > 1.001 mu_0 + 1e-300 (|T_n| <= 1 only on [-1, 1]: spec(H) is not in
 * [a, b]).  Work vectors are taken from the stream-ordered allocator.
 * nb > one kernel row group is processed as column panels. */
chebfd_status chebfd_filter_block(const chebfd_matrix* H, double alpha, double beta,
                                  const double* gc, int Np, void* X, int64_t ld, int nb,
                                  chebfd_dtype vdt, double* moments, void* stream);

/* chebfd_filter_block computed in double-float arithmetic for an FP64 block
 * (vdt C128 or R64 matching H): every entry and matrix value is carried as an
 * unevaluated sum hi + lo of two floats (48-bit significand, unit roundoff
 * ~2^-48 against FP64's 2^-53) and all products and sums use error-free
 * FP32 transformations (TwoSum, FMA TwoProduct) on the paired FP32 pipe,
 * which GB300 executes ~64x faster than FP64.  The block is split into
 * hi/lo panels of 32 complex or 64 real columns, filtered (Fig. ChebFD, the
 * same three step kinds as chebfd_filter_block) and summed back into FP64.
 * Entries must stay inside the FP32 exponent range (|x| < 3e38; the
 * recurrence keeps |T_n(A) x| <= ||x|| while spec(H) lies in [a, b]).
 * Needs a matrix built with also_single (the double-float value copy is built
 * with the FP32 copy).  No moments.  Work panels come from the stream-ordered
 * allocator.  Asynchronous on `stream`.  EINVAL on bad arguments. */
chebfd_status chebfd_filter_block_df(const chebfd_matrix* H, double alpha, double beta,
                                     const double* gc, int Np, void* X, int64_t ld, int nb,
                                     chebfd_dtype vdt, void* stream);

/* Same contract and results as chebfd_filter_block, for callers that cannot
 * allocate device memory at this point: for instance code that runs while
 * another framework owns the device's memory through its own pool (a raw
 * allocation there can fail or split that pool), or a latency-critical loop
 * that must not pay for an allocation or the synchronisation it may imply.
 * The paper has no counterpart of this entry point.
 * The two work vectors and the moment reduction buffers live in one fixed
 * device array of 68 MiB (64 MiB for the work vectors, 4 MiB of moment
 * partials, 256 bytes of counters) that every GPU loading the library keeps
 * until the process exits; the call itself allocates nothing.  Limit: the work
 * vectors need 2 * N * w * element_size <= 64 MiB, where w is the panel
 * width: n_b capped at 32 columns for C128, 64 for C64, 128 for R64 and R32,
 * rounded up to a multiple of 16 bytes.  Examples at the limit: N = 65536
 * with n_b >= 32 C128 or n_b >= 64 C64 (both 16 bytes x 32 or 8 bytes x 64 =
 * 512 bytes per row and vector), N = 65536 with n_b >= 64 R64.  Larger
 * requests return CHEBFD_EINVAL with a message naming the sizes.
 * The first call on a device looks up the device address of the array
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls on a device share the array and it keeps the last call's
 * contents (the counters are cleared on every call): calls whose device work
 * overlaps, from two streams or two host threads, race and must be
 * serialised by the caller.  With moments != NULL the call synchronizes. */
chebfd_status chebfd_filter_block_noalloc(const chebfd_matrix* H, double alpha, double beta,
                                          const double* gc, int Np, void* X, int64_t ld, int nb,
                                          chebfd_dtype vdt, double* moments, void* stream);

/* The filter of chebfd_filter_block (Sec. 2.1, Fig. ChebFD) for a block that
 * lives in HOST memory: X_host (N x nb, row-major, ld >= nb elements per row,
 * rows starting on 16-byte boundaries) is replaced by p[H] X_host.  The block
 * is streamed through the device in panels of the filter's width (C128 32,
 * C64 64, R64/R32 128 columns) with a ring of up to three device panels: the
 * copy of panel p+1 to the device and of panel p-1 back to the host run on
 * two library-owned copy streams while panel p is filtered on `stream`, so
 * the transfers hide behind the filter.  The result equals chebfd_filter_block
 * on a device copy of the block, bit for bit.  X_host should be page-locked
 * (cudaHostAlloc / cudaHostRegister) for the copies to be asynchronous; it is
 * read and written by the device until the work queued on `stream` by this
 * call has completed, and the caller keeps ownership.  Device memory: three
 * panels and two work panels, from the stream-ordered allocator.
 * Errors: CHEBFD_EINVAL for a null or misaligned block, ld < nb, nb < 1,
 * Np < 2 or a dtype that does not match the matrix.  Asynchronous on
 * `stream`. */
chebfd_status chebfd_filter_block_host(const chebfd_matrix* H, double alpha, double beta,
                                       const double* gc, int Np, void* X_host, int64_t ld,
                                       int nb, chebfd_dtype vdt, void* stream);

/* One fused Chebyshev step (Sec. 2.1 recurrence, Fig. ChebFD; the kernel that
 * carries the filter): with U = T_{n-1}(A) X and W = T_{n-2}(A) X on entry,
 * W <- 2(alpha H + beta) U - W = T_n(A) X and Y <- Y + c W in one pass, for
 * device blocks U, W, Y of shape
 * N x nb with a common leading dimension ld (U must not alias W or Y).  nb is
 * limited to one row group (C128/C64: 64, R64/R32: 128 columns).
 * Asynchronous on `stream`. */
chebfd_status chebfd_chebyshev_step(const chebfd_matrix* H, double alpha, double beta, double c,
                                    const void* U, void* W, void* Y, int64_t ld, int nb,
                                    chebfd_dtype vdt, void* stream);

/* -------------------------------------------------------------- KPM (A12) */

/* Normalised KPM moments mu_n = Tr T_n(alpha H + beta) / N, n = 0..M-1, by
 * stochastic trace over R probe vectors (Sec. 3.1 step 1, method of WWAF06):
 * real entries +-1 (bit 0) or complex (+-1 +- i)/sqrt(2) (bits 0, 1) of the
 * SplitMix64 word i*R + r of stream 2.  mu is a HOST array of M doubles, M
 * even, M >= 2.  Synchronizes. */
chebfd_status chebfd_kpm_moments(const chebfd_matrix* H, double alpha, double beta, int M,
                                 int R, uint64_t seed, double* mu, void* stream);

/* Random search block (Sec. 3.1 step 4): X[i*ld + k] = 2u - 1 (real) or
 * (2u - 1) + i(2u' - 1) with u from SplitMix64 stream 1 at word index
 * i*ns_total + (k + col0) (real) or 2*(i*ns_total + k + col0) + {0,1}.
 * Columns col0 .. col0+nb-1 of an ns_total-wide search space. */
chebfd_status chebfd_random_block(void* X, int64_t n, int64_t ld, int nb, int col0,
                                  int ns_total, uint64_t seed, chebfd_dtype vdt, void* stream);

/* ------------------------------------------- orthonormalisation (A7, K3, K5) */

/* Rank-revealing SVQB (Sec. 3.1 step 6; Stathopoulos-Wu) of the device block Y
 * (N x ns, row-major, ld, dtype R64 or C128), in place, all in FP64:
 * S = Y^H Y (cuBLAS HERK/SYRK), D = diag(S)^-1/2, D S D = U Theta U^H
 * (cuSOLVER), directions with Theta_i < ns 2^-52 max Theta dropped and
 * replaced by fresh random vectors (SplitMix64 stream 3; the q-th refill
 * column of the run uses word indices q*N + i, x2 for complex parts, with q
 * continuing from *refill_counter), Y <- Y D U Theta^-1/2; repeated (at most 3
 * passes) while refilled or while max|Y^H Y - I| > 1e-12.  rank (host, may be
 * NULL) receives the rank found in the first pass.  ns <= 1024.  Synchronizes.
 * ENUMERIC if the block has rank 0 or the eigensolver fails. */
chebfd_status chebfd_orthonormalize(void* Y, int64_t n, int ns, int64_t ld, chebfd_dtype vdt,
                                    uint64_t refill_seed, int64_t* refill_counter, int* rank,
                                    void* stream);

/* ---------------------------------------------- Rayleigh-Ritz (A8, K6, K7) */

/* Rayleigh-Ritz step (Sec. 3.1 step 7) for an orthonormal FP64 device block Y
 * (N x ns, ld): G = Y^H (H Y), symmetrised, eigenpairs (theta_k, s_k) in
 * ascending order (cuSOLVER, FP64), Y <- Y S (the Ritz vectors, in place),
 * residual norms res_k = ||H v_k - theta_k v_k|| formed as ||(HY) s_k -
 * theta_k Y s_k|| without a further product with H.  theta[ns] and res[ns] are
 * HOST arrays (res may be NULL); HV (device, N x ns, ld, may be NULL) receives
 * H times the Ritz vectors.  Synchronizes. */
chebfd_status chebfd_rayleigh_ritz(const chebfd_matrix* H, void* Y, int64_t ld, int ns,
                                   chebfd_dtype vdt, double* theta, double* res, void* HV,
                                   void* stream);

/* Harmonic Ritz extraction (the alternative to step 7 named in Sec. 3.1 and
 * Sec. 6; Morgan 1991, Paige-Parlett-van der Vorst 1995) on an ORTHONORMAL
 * device block Y (N x ns, ld, R64/C128) for the target tau (e.g. the window
 * centre): with Z = (H - tau) Y, the Hermitian-definite problem
 * (Y^H Z) s = mu (Z^H Z) s (cuSOLVER, FP64) gives the harmonic Ritz values
 * tau + 1/mu.  In place Y <- the unit harmonic vectors v_k = Y s_k / ||s_k||
 * in ascending order of their Rayleigh quotients theta[k] = v_k^H H v_k
 * (HOST, ns), res[k] = ||H v_k - theta_k v_k|| (HOST, ns, may be NULL),
 * formed from Z and Y without a further product with H.  The vectors are
 * unit but not orthogonal.  If Z^H Z is singular (a column of Y is an exact
 * eigenvector at tau) the ordinary Ritz pairs are returned instead.  EINVAL
 * for a non-finite tau or the block errors of chebfd_rayleigh_ritz.
 * Synchronizes. */
chebfd_status chebfd_harmonic_ritz(const chebfd_matrix* H, void* Y, int64_t ld, int ns,
                                   chebfd_dtype vdt, double tau, double* theta, double* res,
                                   void* stream);

/* res[k] = ||H v_k - theta_k v_k|| (FP64) for the k device vectors V (N x k,
 * ld, R64/C128) and HOST theta[k]; res is a HOST array.  One product with H,
 * per-column sums reduced in a fixed order.  Synchronizes. */
chebfd_status chebfd_residuals(const chebfd_matrix* H, const void* V, const double* theta,
                               int64_t ld, int k, chebfd_dtype vdt, double* res, void* stream);

/* Methods of chebfd_gram. */
typedef enum chebfd_gram_method {
    CHEBFD_GRAM_FP64 = 0,          /* cuBLAS FP64 GEMM (DGEMM / ZGEMM) */
    CHEBFD_GRAM_DOUBLE_FLOAT = 1,  /* the library's double-float kernel on the FP32 pipe */
    CHEBFD_GRAM_TENSOR = 2         /* the library's split onto the bf16 tensor cores */
} chebfd_gram_method;

/* The tall Gram product of the orthonormalisation and Rayleigh-Ritz steps
 * (Sec. 3.1 steps 6-7: S = Y^H Y and Y^H (H Y)): C[p + q m] = sum_i A[i,p]
 * conj(B[i,q]) for device blocks A (N x m, lda) and B (N x m, ldb), row-major,
 * R64 or C128; C is a DEVICE m x m array, column-major (for C128 interleaved
 * complex).  The stored matrix is the complex conjugate of A^H B.
 * CHEBFD_GRAM_TENSOR splits every column of A and B into 8 bf16 digit slices
 * (a power-of-two column scale, a 56-bit fixed-point value, balanced base-128
 * digits; Ozaki, Ogita, Oishi, Rump 2012), multiplies the 36 leading slice
 * pairs with tcgen05.mma, sums the leading digit groups exactly in integers
 * and returns FP64-accurate results (error comparable to an FP64 GEMM);
 * it needs 2 m <= 2048 real columns (m <= 1024 complex) and 16 N m (32 N m
 * complex, twice that when B != A) bytes of workspace from the stream-ordered
 * allocator.  EINVAL on bad arguments; ETIMEOUT if the tensor-core kernel gave
 * up a bounded wait for its pipeline.  Synchronizes. */
chebfd_status chebfd_gram(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n,
                          int m, chebfd_dtype dt, double* C, int method, void* stream);

/* The tall block update of the orthonormalisation and Rayleigh-Ritz steps
 * (Sec. 3.1 steps 6-7: Y <- Y T and the Ritz vectors V = Y S):
 * T[p][i] = sum_q Y[p][q] conj(M[q + i ldm]) for a device block Y (N x k, ldy,
 * row-major) and a DEVICE k x r column-major M (ldm; for C128 interleaved
 * complex), into the device block T (N x r, ldt), R64 or C128; T must not
 * overlap Y.  (M holds the complex conjugate of the transform, the layout in
 * which the Hermitian eigensolvers return column-major eigenvectors of the
 * Gram matrices of chebfd_gram.)  Methods as for chebfd_gram; the tensor
 * method splits every row of Y and every column of M into 8 bf16 digit
 * slices and needs 16 N k (32 N k complex) bytes of workspace; k <= 131072.
 * EINVAL on bad arguments; ETIMEOUT as for chebfd_gram.  Synchronizes. */
chebfd_status chebfd_block_update(const void* Y, int64_t ldy, int64_t n, int k, const double* M,
                                  int ldm, int r, void* T, int64_t ldt, chebfd_dtype dt,
                                  int method, void* stream);

/* Y = X with a change of precision (R64 <-> R32, C128 <-> C64, or a copy);
 * device blocks N x nb with leading dimensions ldx, ldy; round to nearest. */
chebfd_status chebfd_convert_block(const void* X, chebfd_dtype xdt, int64_t ldx, void* Y,
                                   chebfd_dtype ydt, int64_t ldy, int64_t n, int nb,
                                   void* stream);

/* ---------------------------------------------------------- batched ensembles */

/* Ensembles of independent matrices (e.g. disorder realisations of uneven
 * size) filtered together.  The paper filters one matrix; batching many is
 * the same filter (Fig. ChebFD) applied to a block-diagonal matrix.  Members
 * must be built with sell_C = 1, sell_sigma = 1, share one constant row width
 * (13 insulator, 4 graphene) and have dimensions divisible by sell_C; the
 * ensemble stores its own copy (SELL chunk height sell_C), so the members
 * may be destroyed afterwards.  Rows of member i are [off_i, off_{i+1}) of
 * the ensemble; a search block for the ensemble is one row-major
 * N_total x nb device block.  When every member has a blocked copy (see
 * chebfd_matrix_set_blocked) the ensemble concatenates them and its complex64
 * Chebyshev steps run the blocked kernel, bit-identical per member to the
 * member's own filter.  Synchronizes. */
typedef struct chebfd_ensemble chebfd_ensemble;

chebfd_status chebfd_ensemble_create(const chebfd_matrix* const* Hs, int count, int sell_C,
                                     void* stream, chebfd_ensemble** out);

/* n_total, count, row_offsets[count+1] (HOST, may be NULL), SELL chunk
 * height, panel width and row tile of the launches (0 = defaults). */
chebfd_status chebfd_ensemble_info(const chebfd_ensemble* E, int64_t* n_total, int* count,
                                   int64_t* row_offsets, int* sell_C, int* panel, int* tile);

/* Per-member filter coefficients: alpha[count], beta[count] (Eq. W1 for each
 * member's own [a_i, b_i]) and gc[count * (Np+1)] (member i's g_n c_n at
 * gc[i*(Np+1) + n]); all HOST arrays, copied to the device.  Synchronizes. */
chebfd_status chebfd_ensemble_set_coeffs(chebfd_ensemble* E, const double* alpha,
                                         const double* beta, const double* gc, int Np,
                                         void* stream);

/* Launch shape: panel width (columns per fused-step launch) and row tile
 * (consecutive row groups per thread block and wave); 0 = defaults. */
chebfd_status chebfd_ensemble_set_launch(chebfd_ensemble* E, int panel, int tile);

/* X <- p_i[H_i] X on every member's rows at once (Fig. ChebFD with the
 * members' own alpha, beta, g_n c_n): one fused launch per Chebyshev step
 * covers all members.  use_graph != 0 captures the N_p launches once per
 * (X, ld, nb, dtype, N_p, launch shape) into a CUDA graph (instantiated on
 * the first call) and replays it: the whole ensemble filter is one graph
 * launch.  Work vectors are owned by the ensemble.  Asynchronous. */
chebfd_status chebfd_ensemble_filter(chebfd_ensemble* E, void* X, int64_t ld, int nb,
                                     chebfd_dtype vdt, int use_graph, void* stream);

/* Autotuner: builds the ensemble with SELL chunk heights 1, 2, 4 (those
 * dividing every member dimension), times 7 Chebyshev steps on X for each
 * panel width in {16, 32, 48, 64, 128} (admissible for vdt and <= nb) and row
 * tile in {1, 4, 16}, and returns the fastest ensemble with its launch shape
 * set; best_ms (HOST, may be NULL) receives the time per Chebyshev step.  X
 * (N_total x nb, ld) is overwritten.  Synchronizes. */
chebfd_status chebfd_ensemble_autotune(const chebfd_matrix* const* Hs, int count, void* X,
                                       int64_t ld, int nb, chebfd_dtype vdt, void* stream,
                                       chebfd_ensemble** out, double* best_ms);

chebfd_status chebfd_ensemble_destroy(chebfd_ensemble* E);

/* ------------------------------------------- parameter choice (A13, learned) */

/* Features of (H, window) for the parameter-predicting MLP: m_feat normalised
 * KPM moments mu_0..mu_{m_feat-1} of alpha H + beta (1024 moments from 8
 * probe vectors of SplitMix64 stream 2, Sec. 3.1 step 1), then the window
 * centre alpha (lam_lo+lam_hi)/2 + beta, log10 of the scaled half width
 * alpha (lam_hi-lam_lo)/2, and log10 max(N_T, 1) with N_T the KPM count of
 * Eq. DOS:target.  [a, b] with b <= a is computed by chebfd_scale_bounds.
 * features: HOST array of m_feat + 3 doubles; n_target (HOST, may be NULL)
 * receives N_T.  Synchronizes. */
chebfd_status chebfd_param_features(const chebfd_matrix* H, double a, double b, double lam_lo,
                                    double lam_hi, int m_feat, uint64_t seed, double* features,
                                    double* n_target, void* stream);

typedef struct chebfd_mlp chebfd_mlp;

/* (n_s, N_p, kernel) for the window.  mlp == NULL: the paper's rules - N_T
 * from the KPM DOS (Eq. DOS:target), n_s = 4 N_T (Sec. 2.4, linear DOS;
 * Sec. 3.1 step 2) rounded up to a multiple of 8 (>= 16), the margin delta'
 * at which the KPM count reaches n_s (Eq. DOS:search), N_p = N_0 S_w/delta'
 * (Eq. etafit) with N_0 of Tab. lanczoskernel at the window centre, Lanczos
 * kernel.  Otherwise the MLP's outputs (log N_p, log n_s, kernel logit) on the
 * features of chebfd_param_features (m_feat moments), kept inside the range
 * the network was trained on (N_p within [1/2, 2] of the rule's, n_s within
 * [2, 6] N_T).  Either way n_s is never below N_T + 8 rounded up to a
 * multiple of 8 (fewer search vectors than targets cannot converge; the 8
 * covers the KPM estimate's error).  Results are HOST ints; kernel is a
 * chebfd_kernel.  Synchronizes. */
chebfd_status chebfd_choose_params(const chebfd_matrix* H, double a, double b, double lam_lo,
                                   double lam_hi, chebfd_mlp* mlp, int m_feat, uint64_t seed,
                                   int* ns, int* Np, int* kernel, double* n_target,
                                   void* stream);

/* ---------------------------------------------------------------- MLP (K9) */

/* Fully connected network x (n_in) -> tanh (n_hidden) -> tanh (n_hidden) ->
 * 3 outputs (log N_p, log n_s, kernel logit), FP32 on the device, trained
 * and evaluated by this library's kernels.  No counterpart in the paper; the
 * nearest passage is the adaptive choice of N_p and N_S from the DOS
 * suggested in Sec. 6.  Parameters are packed W1 (n_h x n_in, row-major), b1,
 * W2 (n_h x n_h), b2, W3 (3 x n_h), b3; they start at zero. */
chebfd_status chebfd_mlp_create(int n_in, int n_hidden, int n_out, chebfd_mlp** out);
chebfd_status chebfd_mlp_num_params(const chebfd_mlp* N, int64_t* count);
/* Copy packed parameters from HOST floats (resets the Adam state). */
chebfd_status chebfd_mlp_set_params(chebfd_mlp* N, const float* host, int64_t count);
/* Copy packed parameters and/or the last gradient to HOST floats (either may be NULL). */
chebfd_status chebfd_mlp_get_params(const chebfd_mlp* N, float* host, float* host_grads,
                                    int64_t count);
/* Z (DEVICE, B x 3) = network(X (DEVICE, B x n_in, row-major)).  Asynchronous. */
chebfd_status chebfd_mlp_forward(chebfd_mlp* N, const float* X, int B, float* Z, void* stream);
/* Loss (1/B) sum_b [(z0-t0)^2 + (z1-t1)^2 + softplus(z2) - t2 z2] of targets
 * T (DEVICE, B x 3, t2 in {0,1}) and its gradient, kept for chebfd_mlp_adam.
 * loss (HOST, may be NULL; non-NULL synchronizes). */
chebfd_status chebfd_mlp_loss_grad(chebfd_mlp* N, const float* X, const float* T, int B,
                                   float* loss, void* stream);
/* One Adam step (Kingma-Ba) with the last gradient. Asynchronous. */
chebfd_status chebfd_mlp_adam(chebfd_mlp* N, float lr, float beta1, float beta2, float eps,
                              void* stream);
chebfd_status chebfd_mlp_destroy(chebfd_mlp* N);

/* ------------------------------------------------------------- solve (A10) */

typedef enum chebfd_precision {
    CHEBFD_PRECISION_FP64 = 0,  /* FP64 filter, FP64 orthonormalisation and Rayleigh-Ritz */
    CHEBFD_PRECISION_MIXED = 1, /* FP32 / complex64 filter until the residuals stall, then
                                   FP64 filter sweeps; FP64 orthonormalisation, RR, residuals */
    CHEBFD_PRECISION_MIXED_DF = 2 /* as MIXED, but the sweeps after the stall run the
                                   double-float filter (chebfd_filter_block_df) */
} chebfd_precision;

/* Bits of chebfd_params.flags. */
typedef enum chebfd_solve_flags {
    CHEBFD_SOLVE_HARMONIC = 1, /* step 7 with harmonic Ritz pairs for the target
                                 tau = (lam_lo + lam_hi)/2 (chebfd_harmonic_ritz):
                                 window test, ghosts and convergence use their
                                 Rayleigh quotients and residuals; the restart
                                 block is the set of harmonic vectors */
    CHEBFD_SOLVE_LOCKING = 4,  /* hard locking of converged pairs (Sec. 6): an
                                 accepted in-window pair with residual <= eps ||H||
                                 leaves the search block (four at a time, the
                                 smallest residuals first, at least four columns
                                 stay) and is kept as found; every later filtered
                                 block is deflated against the locked vectors
                                 (twice) and the search block shrinks; EINVAL
                                 together with CHEBFD_SOLVE_HARMONIC */
    CHEBFD_SOLVE_ADAPTIVE = 2  /* adaptive degree (Sec. 6 with the rule of Sec. 2.4):
                                 the first filter also returns its Chebyshev
                                 moments; averaged over the n_s random search
                                 vectors (normalised by <x_k, x_k>) they are a
                                 stochastic-trace KPM estimate of the DOS, from
                                 which N_T (Eq. DOS:target), the margin delta'
                                 where the search interval holds n_s states
                                 (Eq. DOS:search) and N_p = N_0 S_w / delta'
                                 (N_0 of Tab. lanczoskernel at the window
                                 centre) follow; that N_p, within [Np/4, 4 Np]
                                 of the given one, is used from the second
                                 iteration on (per-iteration records show it) */
} chebfd_solve_flags;

/* Parameters of chebfd_solve.  Zero / negative fields take the defaults given. */
typedef struct chebfd_params {
    double lam_lo, lam_hi;   /* target interval I_T (closed) */
    double eps;              /* converged if ||H v - theta v|| <= eps * ||H||, ||H|| = max(|a|,|b|) */
    double a, b;             /* spectral interval; b <= a: computed by chebfd_scale_bounds */
    double mu;               /* Lanczos kernel exponent (default 2) */
    int32_t ns;              /* search space size N_S (required, <= 1024) */
    int32_t Np;              /* filter degree N_p (required, >= 2) */
    int32_t kernel;          /* chebfd_kernel (default LANCZOS) */
    int32_t nb;              /* filter panel width (default 64 complex / 128 real) */
    int32_t precision;       /* chebfd_precision */
    int32_t max_iter;        /* default 50 */
    int32_t lanczos_steps;   /* default 30 */
    int32_t flags;           /* chebfd_solve_flags (0: ordinary Ritz pairs); EINVAL for
                                unknown bits; chebfd_solve_batched takes 0 only */
    uint64_t seed;           /* search-vector / refill / Lanczos seed */
    double window_inset;     /* f in [0, 1): the filter's window W = 1 on
                                [c - (1-f) d, c + (1-f) d] inside the target
                                interval [c - d, c + d] (Sec. 2.2: windows with
                                W != 1 on part of I_T); 0 = the rectangular
                                window on I_T.  With the margin d' of the search
                                interval at most d, f = 0.5 lowers the filter's
                                eta (Sec. 2.3) by 20-40% and lets N_p be about
                                halved.  Window test and convergence still use
                                the target interval.  EINVAL outside [0, 1). */
} chebfd_params;

typedef struct chebfd_result chebfd_result;

/* All eigenpairs of H in [lam_lo, lam_hi] by the ChebFD iteration of Sec. 3.1
 * (steps 4-8): random search block (stream 1), then per iteration the filter
 * p[H] of degree Np (chebfd_filter_block), SVQB (chebfd_orthonormalize),
 * Rayleigh-Ritz (chebfd_rayleigh_ritz) and the convergence test.  Ghost Ritz
 * pairs (Sec. 3.1 step 7): from the second iteration on, an in-window pair
 * whose residual exceeds sqrt(eps) ||H|| and did not fall by >= 10x against
 * the previous iteration's pair nearest in theta is discarded.  Converged
 * when at least one pair is accepted and every accepted in-window pair has
 * residual <= eps ||H||, or (empty window) when two successive iterations
 * from the second on have no in-window pair that is accepted or still
 * converging (its residual at most 0.9 of the previous iteration's nearest
 * pair's): ghost-flagged pairs of a weak filter keep converging and keep the
 * iteration going (ENOCONV at max_iter if they never get there), while the
 * in-window Ritz values of a window without eigenvalues stagnate; the
 * restart block is the set of Ritz vectors.
 * MIXED precision switches to FP64 filter sweeps once the largest accepted
 * residual exceeds 1e-9 ||H|| and fell by less than 2x in an iteration.
 * Result handle owned by the library (chebfd_result_destroy).  ENOCONV when
 * max_iter is reached (the result still holds the last iteration).
 * Synchronizes. */
chebfd_status chebfd_solve(const chebfd_matrix* H, const chebfd_params* p, void* stream,
                           chebfd_result** out);

/* Accepted pairs of a result: nev, lambda[nev] (host, ascending), V (device,
 * N x nev row-major FP64: C128 for a complex H, R64 for a real one, ld = nev),
 * res[nev] (host), and the iteration log. Pointers stay valid until destroy. */
typedef struct chebfd_result_info {
    int32_t nev;
    int32_t iterations;
    int32_t converged;
    int32_t fp64_iterations;    /* iterations whose filter ran in FP64 (double-float in MIXED_DF) */
    int64_t n_mvm;              /* products with H (vector count): sum over iterations of N_S N_p */
    double a, b;                /* spectral interval used */
    double seconds_filter, seconds_dense, seconds_total;
    const double* lambda;
    const double* res;
    const void* V;
} chebfd_result_info;

chebfd_status chebfd_result_get(const chebfd_result* r, chebfd_result_info* out);

/* One record per iteration of chebfd_solve (the iteration log of Sec. 3.1
 * steps 5-8, as Fig. ConvTopi tracks it): window and ghost counts of the
 * convergence test, the residual range of the accepted pairs, the precision
 * of the filter, and where the time went.  The dense seconds are CUDA-event
 * times on the solve's stream, split into the tall Gram products (Y^H Y,
 * Y^H H Y, and Z^H Z with harmonic pairs), the tall block products (Y T,
 * Ritz vectors, H V), the n_s x n_s eigenproblems with their small products
 * and host decisions, the products H Y, the residual norms, and anything
 * else (the separate-call path after a rank drop). */
typedef struct chebfd_iteration_info {
    int32_t iteration;          /* 1-based */
    int32_t fp64_filter;        /* 1: the filter ran in FP64 (double-float in MIXED_DF), 0: single */
    int32_t in_window;          /* Ritz values in [lam_lo, lam_hi] */
    int32_t ghosts;             /* of them ghost-flagged */
    int32_t accepted;           /* in-window pairs accepted (not ghosts) */
    int32_t converged_pairs;    /* accepted pairs with residual <= eps ||H|| */
    int32_t Np;                 /* degree of this iteration's filter */
    int32_t locked;             /* pairs locked before this iteration (CHEBFD_SOLVE_LOCKING) */
    double res_min, res_max;    /* over the accepted pairs, absolute; -1 when none */
    double seconds_filter;      /* host wall time of the filter (stream synchronized) */
    double seconds_dense;       /* host wall time of steps 6-7 */
    double seconds_gram, seconds_block_gemm, seconds_eigensolve, seconds_hy,
        seconds_residuals, seconds_other;
} chebfd_iteration_info;

/* Copy up to `capacity` iteration records of a chebfd_solve result into the
 * HOST array out (may be NULL when capacity is 0); *count (HOST) receives the
 * number of records (= info.iterations).  Results of chebfd_solve_batched
 * carry records with the counts and residuals but zero seconds. */
chebfd_status chebfd_result_iterations(const chebfd_result* r, chebfd_iteration_info* out,
                                       int capacity, int* count);

/* Copy the accepted Ritz vectors (N x nev) into the caller's DEVICE buffer dst
 * (row-major, leading dimension ld >= nev, same FP64 type as the result).
 * Synchronizes `stream`. */
chebfd_status chebfd_result_copy_vectors(const chebfd_result* r, void* dst, int64_t ld,
                                         void* stream);

chebfd_status chebfd_result_destroy(chebfd_result* r);

/* chebfd_solve for every member of an ensemble at once (one ensemble filter
 * per iteration, one CUDA-graph launch; SVQB and Rayleigh-Ritz member by
 * member on their row slices; the convergence and ghost rules of
 * chebfd_solve per member).  Hs[count] are the member matrices the ensemble
 * was built from (used for H V in the projection), a[count], b[count] their
 * spectral intervals (HOST), p the common window, eps, ns, Np, kernel, mu,
 * precision, max_iter and seed (p->a, p->b, p->nb, p->lanczos_steps
 * ignored).  MIXED precision filters in single precision until every
 * unconverged member has stalled, then in FP64.  outs[count] receive one
 * result per member (converged or not; destroy each).  iterations (HOST, may
 * be NULL) receives the iterations run.  Synchronizes. */
chebfd_status chebfd_solve_batched(chebfd_ensemble* E, const chebfd_matrix* const* Hs,
                                   const double* a, const double* b, const chebfd_params* p,
                                   void* stream, chebfd_result** outs, int* iterations);

#ifdef __cplusplus
}
#endif

#endif /* CHEBFD_H */
