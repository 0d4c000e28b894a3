// Device-side matrix construction: lattice Hamiltonian generators (CSR) and
// the SELL-C-sigma build (Sec. 4; format of Kreutzer et al. 2014).
#include <cub/cub.cuh>
#include <cstdlib>

#include "common.cuh"

namespace chebfd {

namespace {

struct Entry {
    int64_t col;
    double re, im;
    int order;
};

struct LatticeParams {
    int kind;
    int64_t Lx, Ly, Lz;
    double t, m, W;
    uint64_t seed;
};

constexpr int MAX_CONTRIB = 13;

// Contributions of one row in the fixed order onsite, +x, -x, +y, -y, +z, -z.
__device__ int topi_contributions(int64_t row, const LatticeParams& P, Entry* e) {
    const int64_t s = row >> 2;
    const int o = (int)(row & 3);
    const int64_t x = s % P.Lx, y = (s / P.Lx) % P.Ly, z = s / (P.Lx * P.Ly);
    const double u = splitmix_uniform(P.seed, STREAM_DISORDER, (uint64_t)s);
    const double V = __dmul_rn(P.W, u - 0.5);
    const double h = P.t / 2.0;
    const bool upper = o < 2;  // Gamma1 = diag(1, 1, -1, -1)
    const bool slab = P.kind == CHEBFD_LATTICE_TOPI_SLAB;
    // onsite: (m + V_s) Gamma1, or for the slab V_s Gamma0 + m Gamma1 (Eq. Ham)
    double onsite;
    if (slab)
        onsite = upper ? __dadd_rn(V, P.m) : __dadd_rn(V, -P.m);
    else
        onsite = upper ? __dadd_rn(P.m, V) : -__dadd_rn(P.m, V);
    int c = 0;
    e[c++] = Entry{4 * s + o, onsite, 0.0, 0};
    int rank = 1;
    for (int j = 0; j < 3; ++j) {
        // Off-diagonal partner p of Gamma_{j+1} and the entry Gamma_{j+1}[o][p].
        int p;
        double gr = 0.0, gi = 0.0;
        if (j == 0) {  // sx (x) sx: (0,3),(1,2),(2,1),(3,0) = 1
            p = o ^ 3;
            gr = 1.0;
        } else if (j == 1) {  // sx (x) sy: (0,3) = -i, (1,2) = i, (2,1) = -i, (3,0) = i
            p = o ^ 3;
            gi = (o == 0 || o == 2) ? -1.0 : 1.0;
        } else {  // sx (x) sz: (0,2) = 1, (1,3) = -1, (2,0) = 1, (3,1) = -1
            p = o ^ 2;
            gr = (o == 0 || o == 2) ? 1.0 : -1.0;
        }
        for (int sg = 0; sg < 2; ++sg) {
            const int64_t sign = sg == 0 ? 1 : -1;
            int64_t cx = x, cy = y, cz = z;
            if (j == 0) cx = (x + sign + P.Lx) % P.Lx;
            if (j == 1) cy = (y + sign + P.Ly) % P.Ly;
            if (j == 2) {
                if (slab && (z + sign < 0 || z + sign >= P.Lz)) continue;  // open in z
                cz = (z + sign + P.Lz) % P.Lz;
            }
            const int64_t sn = cx + P.Lx * (cy + P.Ly * cz);
            const double dval = upper ? -h : h;  // -h * Gamma1[o][o]
            const double q = sign < 0 ? 1.0 : -1.0;  // T_j at s-e_j, T_j^dagger at s+e_j
            const double ore = __dadd_rn(__dmul_rn(-q * h, gi), 0.0);
            const double oim = __dadd_rn(__dmul_rn(q * h, gr), 0.0);
            e[c++] = Entry{4 * sn + o, dval, 0.0, rank++};
            e[c++] = Entry{4 * sn + p, ore, oim, rank++};
        }
    }
    return c;
}

__device__ int graphene_contributions(int64_t row, const LatticeParams& P, Entry* e) {
    const int64_t cell = row >> 1;
    const int sub = (int)(row & 1);
    const int64_t i = cell % P.Lx, j = cell / P.Lx;
    const double u = splitmix_uniform(P.seed, STREAM_DISORDER, (uint64_t)row);
    const double V = __dmul_rn(P.W, u - 0.5);
    int c = 0;
    e[c++] = Entry{row, V, 0.0, 0};
    int64_t nb[3];
    if (sub == 0) {  // A(i,j): B(i,j), B(i-1,j), B(i,j-1)
        nb[0] = i + P.Lx * j;
        nb[1] = (i - 1 + P.Lx) % P.Lx + P.Lx * j;
        nb[2] = i + P.Lx * ((j - 1 + P.Ly) % P.Ly);
    } else {  // B(i,j): A(i,j), A(i+1,j), A(i,j+1)
        nb[0] = i + P.Lx * j;
        nb[1] = (i + 1) % P.Lx + P.Lx * j;
        nb[2] = i + P.Lx * ((j + 1) % P.Ly);
    }
    for (int k = 0; k < 3; ++k) e[c++] = Entry{2 * nb[k] + (1 - sub), -P.t, 0.0, k + 1};
    return c;
}

// Stable sort by column, then merge equal columns summing left to right.
__device__ int row_entries(int64_t row, const LatticeParams& P, Entry* e) {
    int c = P.kind == CHEBFD_LATTICE_GRAPHENE ? graphene_contributions(row, P, e)
                                              : topi_contributions(row, P, e);
    for (int a = 1; a < c; ++a) {
        Entry v = e[a];
        int b = a - 1;
        while (b >= 0 && e[b].col > v.col) {
            e[b + 1] = e[b];
            --b;
        }
        e[b + 1] = v;
    }
    int out = 0;
    for (int a = 0; a < c;) {
        Entry acc = e[a];
        int b = a + 1;
        while (b < c && e[b].col == acc.col) {
            acc.re = __dadd_rn(acc.re, e[b].re);
            acc.im = __dadd_rn(acc.im, e[b].im);
            ++b;
        }
        e[out++] = acc;
        a = b;
    }
    return out;
}

__global__ void lattice_count_kernel(LatticeParams P, int64_t n, int64_t* rowlen) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        Entry e[MAX_CONTRIB];
        rowlen[r + 1] = row_entries(r, P, e);
        if (r == 0) rowlen[0] = 0;
    }
}

__global__ void lattice_fill_kernel(LatticeParams P, int64_t n, const int64_t* rowptr,
                                    int32_t* col, double* val, bool cplx) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        Entry e[MAX_CONTRIB];
        int c = row_entries(r, P, e);
        int64_t base = rowptr[r];
        for (int k = 0; k < c; ++k) {
            col[base + k] = (int32_t)e[k].col;
            if (cplx) {
                val[2 * (base + k)] = e[k].re;
                val[2 * (base + k) + 1] = e[k].im;
            } else {
                val[base + k] = e[k].re;
            }
        }
    }
}

__global__ void rowlen_kernel(const int64_t* rowptr, int64_t n, int32_t* len) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        len[r] = (int32_t)(rowptr[r + 1] - rowptr[r]);
}

__global__ void sort_keys_kernel(const int32_t* len, int64_t n, int64_t sigma, uint64_t* key,
                                 int64_t* idx) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        uint64_t w = (uint64_t)(r / sigma);
        key[r] = (w << 32) | (uint64_t)(0x7FFFFFFFu - (uint32_t)len[r]);
        idx[r] = r;
    }
}

__global__ void identity_perm_kernel(int64_t* perm, int64_t n) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        perm[r] = r;
}

__global__ void chunk_len_kernel(const int32_t* len, const int64_t* perm, int64_t n, int C,
                                 int64_t nchunks, int32_t* chunk_len, int64_t* chunk_slots) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nchunks;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = 0;
        for (int l = 0; l < C; ++l) {
            int64_t r = k * C + l;
            if (r < n) m = max(m, len[perm[r]]);
        }
        chunk_len[k] = m;
        chunk_slots[k] = (int64_t)m * C;
    }
}

template <bool CPLX>
__global__ void sell_fill_kernel(const int64_t* rowptr, const int32_t* ccol, const double* cval,
                                 const int64_t* perm, const int64_t* chunk_ptr,
                                 const int32_t* chunk_len, int64_t n, int C, int64_t nchunks,
                                 int32_t* scol, double* sval) {
    const int64_t rows = nchunks * C;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = r / C;
        const int l = (int)(r % C);
        const int64_t base = chunk_ptr[k] + l;
        const int len = chunk_len[k];
        int64_t b = 0, e = 0, orig = 0;
        if (r < n) {
            orig = perm[r];
            b = rowptr[orig];
            e = rowptr[orig + 1];
        }
        for (int j = 0; j < len; ++j) {
            const int64_t pos = base + (int64_t)j * C;
            if (j < e - b) {
                scol[pos] = ccol[b + j];
                if (CPLX) {
                    sval[2 * pos] = cval[2 * (b + j)];
                    sval[2 * pos + 1] = cval[2 * (b + j) + 1];
                } else {
                    sval[pos] = cval[b + j];
                }
            } else {
                scol[pos] = (int32_t)orig;
                if (CPLX) {
                    sval[2 * pos] = 0.0;
                    sval[2 * pos + 1] = 0.0;
                } else {
                    sval[pos] = 0.0;
                }
            }
        }
    }
}

__global__ void to_df_values_kernel(const double* v, float2* d, int64_t count) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x) {
        const float hi = __double2float_rn(v[t]);
        d[t] = make_float2(hi, __double2float_rn(v[t] - (double)hi));
    }
}

__global__ void to_single_kernel(const double* in, float* out, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __double2float_rn(in[i]);
}

int grid_for(int64_t work, int threads = 256) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65535 * 16) g = 65535 * 16;
    return (int)g;
}

// ------------------------------------------------------------ blocked ELL copy

// Block columns of block row br other than br itself, ascending and distinct,
// into list[0 .. kBellLB-2]; returns their count, or kBellLB when there are
// more than kBellLB - 1 (the matrix then gets no blocked copy).
__device__ int bell_collect(const int64_t* rowptr, const int32_t* ccol, int64_t br,
                            int32_t* list) {
    int cnt = 0;
    for (int r = 0; r < kBellB; ++r) {
        const int64_t row = br * kBellB + r;
        for (int64_t p = rowptr[row]; p < rowptr[row + 1]; ++p) {
            const int32_t bc = ccol[p] / kBellB;
            if (bc == br) continue;
            int i = 0;
            while (i < cnt && list[i] < bc) ++i;
            if (i < cnt && list[i] == bc) continue;
            if (cnt == kBellLB - 1) return kBellLB;
            for (int j = cnt; j > i; --j) list[j] = list[j - 1];
            list[i] = bc;
            ++cnt;
        }
    }
    return cnt;
}

__global__ void bell_check_kernel(const int64_t* rowptr, const int32_t* ccol, int64_t nbr,
                                  int* too_many) {
    for (int64_t br = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; br < nbr;
         br += (int64_t)gridDim.x * blockDim.x) {
        int32_t list[kBellLB];
        if (bell_collect(rowptr, ccol, br, list) >= kBellLB) atomicOr(too_many, 1);
    }
}

// Slot 0 holds the diagonal block, slots 1.. the other block columns in
// ascending order, unused slots the diagonal block again with zero values.
// Repeated (row, column) entries are summed in FP64 before rounding.
__global__ void bell_fill_kernel(const int64_t* rowptr, const int32_t* ccol, const double* cval,
                                 int64_t nbr, int32_t* bcol, float2* bval) {
    for (int64_t br = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; br < nbr;
         br += (int64_t)gridDim.x * blockDim.x) {
        int32_t list[kBellLB];
        const int cnt = bell_collect(rowptr, ccol, br, list);
        int32_t cols[kBellLB];
        cols[0] = (int32_t)br;
        for (int k = 1; k < kBellLB; ++k) cols[k] = k - 1 < cnt ? list[k - 1] : (int32_t)br;
        double2 acc[kBellLB][kBellB * kBellB];
        for (int k = 0; k < kBellLB; ++k)
            for (int e = 0; e < kBellB * kBellB; ++e) acc[k][e] = make_double2(0.0, 0.0);
        for (int r = 0; r < kBellB; ++r) {
            const int64_t row = br * kBellB + r;
            for (int64_t p = rowptr[row]; p < rowptr[row + 1]; ++p) {
                const int32_t c = ccol[p];
                const int32_t bc = c / kBellB;
                int k = 0;
                if (bc != br)
                    for (k = 1; k < kBellLB && cols[k] != bc; ++k) {
                    }
                if (k == kBellLB) continue;  // not reached: every block column was collected
                double2& a = acc[k][r * kBellB + (c - bc * kBellB)];
                a.x += cval[2 * p];
                a.y += cval[2 * p + 1];
            }
        }
        for (int k = 0; k < kBellLB; ++k) {
            bcol[br * kBellLB + k] = cols[k];
            for (int e = 0; e < kBellB * kBellB; ++e) {
                const int64_t q = (br * kBellLB + k) * (kBellB * kBellB) + e;
                bval[q] = make_float2(__double2float_rn(acc[k][e].x),
                                      __double2float_rn(acc[k][e].y));
            }
        }
    }
}

}  // namespace

void generate_lattice_csr(const chebfd_lattice_desc& d, int64_t* n_out, int64_t** d_rowptr,
                          int32_t** d_col, void** d_val, cudaStream_t stream) {
    CHEBFD_REQUIRE(d.kind == CHEBFD_LATTICE_TOPI || d.kind == CHEBFD_LATTICE_GRAPHENE ||
                       d.kind == CHEBFD_LATTICE_TOPI_SLAB,
                   CHEBFD_EINVAL, "unknown lattice kind");
    CHEBFD_REQUIRE(d.Lx >= 1 && d.Ly >= 1 && (d.kind == CHEBFD_LATTICE_GRAPHENE || d.Lz >= 1),
                   CHEBFD_EINVAL, "lattice edges must be >= 1");
    CHEBFD_REQUIRE(d.seed < (1ULL << 56), CHEBFD_EINVAL, "seed must be < 2^56");
    LatticeParams P;
    P.kind = d.kind;
    P.Lx = d.Lx;
    P.Ly = d.Ly;
    const bool topi = d.kind != CHEBFD_LATTICE_GRAPHENE;
    P.Lz = topi ? d.Lz : 1;
    P.t = d.t;
    P.m = d.m;
    P.W = d.W;
    P.seed = d.seed;
    const int64_t n = topi ? 4 * P.Lx * P.Ly * P.Lz : 2 * P.Lx * P.Ly;
    CHEBFD_REQUIRE(n < (1LL << 31), CHEBFD_EINVAL, "matrix dimension must be < 2^31");
    const bool cplx = topi;
    int64_t *rowptr = nullptr, *counts = nullptr;
    CHEBFD_CHECK_CUDA(cudaMalloc(&rowptr, (n + 1) * sizeof(int64_t)));
    CHEBFD_CHECK_CUDA(cudaMalloc(&counts, (n + 1) * sizeof(int64_t)));
    lattice_count_kernel<<<grid_for(n), 256, 0, stream>>>(P, n, counts);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
    size_t tmp_bytes = 0;
    cub::DeviceScan::InclusiveSum(nullptr, tmp_bytes, counts, rowptr, n + 1, stream);
    void* tmp = nullptr;
    CHEBFD_CHECK_CUDA(cudaMalloc(&tmp, tmp_bytes));
    cub::DeviceScan::InclusiveSum(tmp, tmp_bytes, counts, rowptr, n + 1, stream);
    int64_t nnz = 0;
    CHEBFD_CHECK_CUDA(
        cudaMemcpyAsync(&nnz, rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(stream));
    cudaFree(tmp);
    cudaFree(counts);
    int32_t* col = nullptr;
    double* val = nullptr;
    CHEBFD_CHECK_CUDA(cudaMalloc(&col, nnz * sizeof(int32_t)));
    CHEBFD_CHECK_CUDA(cudaMalloc(&val, nnz * sizeof(double) * (cplx ? 2 : 1)));
    lattice_fill_kernel<<<grid_for(n), 256, 0, stream>>>(P, n, rowptr, col, val, cplx);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
    *n_out = n;
    *d_rowptr = rowptr;
    *d_col = col;
    *d_val = val;
}

void build_sell_from_device_csr(Matrix& M, const int64_t* rowptr, const int32_t* ccol,
                                const void* cval, int C, int sigma, bool also_single,
                                cudaStream_t stream) {
    const int64_t n = M.n;
    CHEBFD_REQUIRE(C >= 1 && C <= 32 && (C & (C - 1)) == 0, CHEBFD_EINVAL,
                   "SELL chunk height C must be a power of two in [1, 32]");
    CHEBFD_REQUIRE(sigma >= 1, CHEBFD_EINVAL, "SELL sigma must be >= 1");
    M.C = C;
    M.sigma = sigma;
    M.nchunks = (n + C - 1) / C;
    int32_t* len = nullptr;
    CHEBFD_CHECK_CUDA(cudaMalloc(&len, n * sizeof(int32_t)));
    rowlen_kernel<<<grid_for(n), 256, 0, stream>>>(rowptr, n, len);
    CHEBFD_CHECK_CUDA(cudaMalloc(&M.perm, n * sizeof(int64_t)));
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    if (sigma > 1) {
        uint64_t *keys = nullptr, *keys_out = nullptr;
        int64_t* idx = nullptr;
        CHEBFD_CHECK_CUDA(cudaMalloc(&keys, n * sizeof(uint64_t)));
        CHEBFD_CHECK_CUDA(cudaMalloc(&keys_out, n * sizeof(uint64_t)));
        CHEBFD_CHECK_CUDA(cudaMalloc(&idx, n * sizeof(int64_t)));
        sort_keys_kernel<<<grid_for(n), 256, 0, stream>>>(len, n, sigma, keys, idx);
        // LSD radix sort is stable: equal keys keep ascending original index.
        cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys, keys_out, idx, M.perm, n, 0,
                                        64, stream);
        CHEBFD_CHECK_CUDA(cudaMalloc(&tmp, tmp_bytes));
        cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys, keys_out, idx, M.perm, n, 0, 64,
                                        stream);
        CHEBFD_CHECK_CUDA(cudaStreamSynchronize(stream));
        cudaFree(tmp);
        cudaFree(keys);
        cudaFree(keys_out);
        cudaFree(idx);
        tmp = nullptr;
        M.identity_perm = false;
    } else {
        identity_perm_kernel<<<grid_for(n), 256, 0, stream>>>(M.perm, n);
        M.identity_perm = true;
    }
    CHEBFD_CHECK_CUDA(cudaMalloc(&M.chunk_len, M.nchunks * sizeof(int32_t)));
    CHEBFD_CHECK_CUDA(cudaMalloc(&M.chunk_ptr, (M.nchunks + 1) * sizeof(int64_t)));
    int64_t* slots = nullptr;
    CHEBFD_CHECK_CUDA(cudaMalloc(&slots, M.nchunks * sizeof(int64_t)));
    chunk_len_kernel<<<grid_for(M.nchunks), 256, 0, stream>>>(len, M.perm, n, C, M.nchunks,
                                                               M.chunk_len, slots);
    CHEBFD_CHECK_CUDA(cudaMemsetAsync(M.chunk_ptr, 0, sizeof(int64_t), stream));
    tmp_bytes = 0;
    cub::DeviceScan::InclusiveSum(nullptr, tmp_bytes, slots, M.chunk_ptr + 1, M.nchunks, stream);
    size_t tmp2 = 0;
    cub::DeviceReduce::Max(nullptr, tmp2, len, len, n, stream);
    tmp_bytes = std::max(tmp_bytes, tmp2);
    CHEBFD_CHECK_CUDA(cudaMalloc(&tmp, tmp_bytes + 64));
    cub::DeviceScan::InclusiveSum(tmp, tmp_bytes, slots, M.chunk_ptr + 1, M.nchunks, stream);
    int32_t* dmax = nullptr;
    CHEBFD_CHECK_CUDA(cudaMalloc(&dmax, sizeof(int32_t)));
    size_t tb = tmp_bytes;
    cub::DeviceReduce::Max(tmp, tb, len, dmax, n, stream);
    int64_t total = 0;
    int32_t maxlen = 0;
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(&total, M.chunk_ptr + M.nchunks, sizeof(int64_t),
                                      cudaMemcpyDeviceToHost, stream));
    CHEBFD_CHECK_CUDA(
        cudaMemcpyAsync(&maxlen, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    int64_t nnz = 0;
    CHEBFD_CHECK_CUDA(
        cudaMemcpyAsync(&nnz, rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(stream));
    cudaFree(tmp);
    cudaFree(dmax);
    cudaFree(slots);
    M.nnz_padded = total;
    M.nnz = nnz;
    M.max_row_len = maxlen;
    // every chunk has the widest row's width exactly when the slot count says so
    M.uniform_width = (total == M.nchunks * (int64_t)C * maxlen) ? maxlen : 0;
    const size_t vsz = M.complex_values ? 16 : 8;
    CHEBFD_CHECK_CUDA(cudaMalloc(&M.col, std::max<int64_t>(total, 1) * sizeof(int32_t)));
    CHEBFD_CHECK_CUDA(cudaMalloc(&M.val64, std::max<int64_t>(total, 1) * vsz));
    const int64_t rows = M.nchunks * C;
    if (M.complex_values)
        sell_fill_kernel<true><<<grid_for(rows), 256, 0, stream>>>(
            rowptr, ccol, (const double*)cval, M.perm, M.chunk_ptr, M.chunk_len, n, C, M.nchunks,
            M.col, (double*)M.val64);
    else
        sell_fill_kernel<false><<<grid_for(rows), 256, 0, stream>>>(
            rowptr, ccol, (const double*)cval, M.perm, M.chunk_ptr, M.chunk_len, n, C, M.nchunks,
            M.col, (double*)M.val64);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
    if (also_single) {
        const int64_t count = total * (M.complex_values ? 2 : 1);
        CHEBFD_CHECK_CUDA(cudaMalloc(&M.val32, std::max<int64_t>(count, 1) * sizeof(float)));
        to_single_kernel<<<grid_for(count), 256, 0, stream>>>((const double*)M.val64,
                                                              (float*)M.val32, count);
        CHEBFD_CHECK_CUDA(cudaGetLastError());
        // double-float copy: each FP64 value v -> (hi, lo) = (fl32(v), fl32(v - hi))
        CHEBFD_CHECK_CUDA(cudaMalloc(&M.valdf, std::max<int64_t>(count, 1) * 2 * sizeof(float)));
        to_df_values_kernel<<<grid_for(count), 256, 0, stream>>>((const double*)M.val64,
                                                                (float2*)M.valdf, count);
        CHEBFD_CHECK_CUDA(cudaGetLastError());
    }
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(stream));
    cudaFree(len);
    if (also_single && M.complex_values && M.identity_perm && n % kBellB == 0) {
        const char* e = getenv("CHEBFD_BLOCKED");
        if (!(e && e[0] == '0')) build_bell(M, rowptr, ccol, (const double*)cval, stream);
    }
}

void build_bell(Matrix& M, const int64_t* rowptr, const int32_t* ccol, const double* cval,
                cudaStream_t stream) {
    const int64_t nbr = M.n / kBellB;
    // dense blocks may store at most 4x the entries they replace
    if (nbr == 0 || (double)kBellLB * kBellB * kBellB > 4.0 * (double)M.nnz / (double)nbr) return;
    int* flag = nullptr;
    CHEBFD_CHECK_CUDA(cudaMalloc(&flag, sizeof(int)));
    CHEBFD_CHECK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), stream));
    bell_check_kernel<<<grid_for(nbr), 256, 0, stream>>>(rowptr, ccol, nbr, flag);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
    int too_many = 0;
    CHEBFD_CHECK_CUDA(cudaMemcpyAsync(&too_many, flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(stream));
    cudaFree(flag);
    if (too_many) return;
    CHEBFD_CHECK_CUDA(cudaMalloc(&M.bell_col, nbr * kBellLB * sizeof(int32_t)));
    CHEBFD_CHECK_CUDA(
        cudaMalloc(&M.bell_val32, nbr * kBellLB * kBellB * kBellB * sizeof(float2)));
    bell_fill_kernel<<<grid_for(nbr, 128), 128, 0, stream>>>(rowptr, ccol, cval, nbr, M.bell_col,
                                                            (float2*)M.bell_val32);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
    CHEBFD_CHECK_CUDA(cudaStreamSynchronize(stream));
    M.bell_enabled = true;
}

}  // namespace chebfd
