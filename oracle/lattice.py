"""Test matrices of the paper's workloads as CSR (oracle side).

* Topological insulator (Eq. Ham, Sec. 5.1), in the configuration form used by
  this project's workloads: onsite block (m + V_s) Gamma1, hopping from site s
  to s + e_j given by the block T_j = -(t/2)(Gamma1 - i Gamma_{j+1}) at
  (row of s + e_j, column of s) plus its Hermitian conjugate at the transposed
  position; periodic in all three axes; 4 orbitals per site; row = 4 s + o with
  s = x + Lx (y + Ly z).  This gives the 13 stored entries per row quoted in
  Sec. 4 (N_nzr = 13).
* The paper's own form of Eq. Ham (`topi_slab_csr`): the same hopping, onsite
  V_n Gamma^0 + m Gamma^1 with Gamma^0 the identity (m = 2 in Sec. 5.1), on a
  slab that is periodic in x and y and open in z (the surface layers have no
  z neighbour outside the slab: 11 entries in their rows).
* Graphene (Sec. 5.4, Tab. benchmark): honeycomb lattice, hopping -t between
  nearest neighbours, onsite disorder; 4 stored entries per row with the
  diagonal (N_nzr = 4 in Sec. 4).
* Diagonal matrices with flat DOS (Sec. 2.2: lambda_i = -1 + 2 i / (D+1)) and
  with linear DOS rho = rho_1 |lambda| (Sec. 2.4, Tab. num).

Disorder V = W (u - 1/2) with u from SplitMix64 stream 0 (one value per site for
the insulator, per atom for graphene).  Columns are ascending within a row;
entries that land on the same (row, column) - only on lattices with an edge
of length 1 or 2 - are summed left to right in the fixed contribution order
(onsite, +x, -x, +y, -y, +z, -z).  Every structural entry is stored, zeros
included.
"""
import numpy as np
import scipy.sparse as sp

from . import rng

# Dirac matrices Gamma1..Gamma4 as Kronecker products of Pauli matrices.
_S0 = np.eye(2, dtype=np.complex128)
_SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
GAMMA = [np.kron(_SZ, _S0), np.kron(_SX, _SX), np.kron(_SX, _SY), np.kron(_SX, _SZ)]


def _merge(rows, cols, vals, order, n, dtype):
    """Sort contributions by (row, col, order) and sum duplicates in order."""
    key = np.lexsort((order, cols, rows))
    rows, cols, vals = rows[key], cols[key], vals[key]
    same = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
    if same.any():
        out_r, out_c, out_v = [], [], []
        i = 0
        m = len(rows)
        while i < m:
            acc = vals[i]
            j = i + 1
            while j < m and rows[j] == rows[i] and cols[j] == cols[i]:
                acc = acc + vals[j]
                j += 1
            out_r.append(rows[i]); out_c.append(cols[i]); out_v.append(acc)
            i = j
        rows = np.array(out_r, dtype=np.int64)
        cols = np.array(out_c, dtype=np.int64)
        vals = np.array(out_v, dtype=dtype)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cols.astype(np.int32), vals.astype(dtype)


def disorder(seed, count, W):
    """V_k = W (u_k - 1/2), u from stream 0 at index k."""
    u = rng.uniform(seed, rng.STREAM_DISORDER, np.arange(count, dtype=np.uint64))
    return W * (u - 0.5)


def topi_csr(Lx, Ly, Lz, t=1.0, m=1.0, W=0.0, seed=0, sites=None):
    """CSR (rowptr int64, col int32, val complex128) of the insulator Hamiltonian.
    With `sites` (an int64 array of site indices) only the 4 rows of each
    listed site are generated: the CSR then has 4 len(sites) rows, row 4 q + o
    being row 4 sites[q] + o of the full matrix (columns stay global)."""
    nsite_all = Lx * Ly * Lz
    s = np.arange(nsite_all, dtype=np.int64) if sites is None else np.asarray(sites, np.int64)
    nsite = len(s)
    n = 4 * nsite
    x = s % Lx
    y = (s // Lx) % Ly
    z = s // (Lx * Ly)
    V = disorder(seed, nsite_all, W)[s] if sites is None else W * (
        rng.uniform(seed, rng.STREAM_DISORDER, s.astype(np.uint64)) - 0.5)
    mv = m + V                                   # one rounding per site
    h = t / 2.0
    rows, cols, vals, order = [], [], [], []
    g1 = np.real(np.diag(GAMMA[0]))              # +1, +1, -1, -1
    q_local = np.arange(nsite, dtype=np.int64)
    for o in range(4):
        r = 4 * q_local + o                      # local row (= global row for the full matrix)
        # onsite (m + V_s) Gamma1
        rows.append(r); cols.append(4 * s + o)
        vals.append((mv if g1[o] > 0 else -mv).astype(np.complex128))
        order.append(np.zeros(nsite, dtype=np.int64))
        rank = 1
        for j, L in enumerate((Lx, Ly, Lz)):
            G = GAMMA[j + 1]
            p = int(np.nonzero(G[o])[0][0])        # off-diagonal column of Gamma_{j+1}
            for sign in (+1, -1):
                cx, cy, cz = x.copy(), y.copy(), z.copy()
                if j == 0:
                    cx = (x + sign) % Lx
                elif j == 1:
                    cy = (y + sign) % Ly
                else:
                    cz = (z + sign) % Lz
                sn = cx + Lx * (cy + Ly * cz)
                # column site s+e_j carries T_j^dagger, column site s-e_j carries T_j;
                # off-diagonal entry q i h Gamma[o,p] (q = +1 for T_j, -1 for T_j^dagger)
                # written out in real arithmetic, zeros as +0.0
                dval = -h * g1[o]
                q = 1.0 if sign < 0 else -1.0
                off = complex(-q * h * G[o, p].imag + 0.0, q * h * G[o, p].real + 0.0)
                rows.append(r); cols.append(4 * sn + o)
                vals.append(np.full(nsite, dval, dtype=np.complex128))
                order.append(np.full(nsite, rank, dtype=np.int64)); rank += 1
                rows.append(r); cols.append(4 * sn + p)
                vals.append(np.full(nsite, off, dtype=np.complex128))
                order.append(np.full(nsite, rank, dtype=np.int64)); rank += 1
    rows = np.concatenate(rows); cols = np.concatenate(cols)
    vals = np.concatenate(vals); order = np.concatenate(order)
    return _merge(rows, cols, vals, order, n, np.complex128)


def topi_slab_csr(Lx, Ly, Lz, t=1.0, m=2.0, W=0.0, seed=0):
    """CSR of Eq. Ham on an Lx x Ly x Lz slab (periodic in x, y; open in z):
    onsite V_s + m Gamma1[o][o] on the diagonal, hopping as in topi_csr."""
    nsite = Lx * Ly * Lz
    n = 4 * nsite
    s = np.arange(nsite, dtype=np.int64)
    x = s % Lx
    y = (s // Lx) % Ly
    z = s // (Lx * Ly)
    V = disorder(seed, nsite, W)
    h = t / 2.0
    rows, cols, vals, order = [], [], [], []
    g1 = np.real(np.diag(GAMMA[0]))
    for o in range(4):
        r = 4 * s + o
        rows.append(r); cols.append(4 * s + o)
        vals.append((V + m * g1[o]).astype(np.complex128))   # one rounding: V + m or V - m
        order.append(np.zeros(nsite, dtype=np.int64))
        rank = 1
        for j in range(3):
            G = GAMMA[j + 1]
            p = int(np.nonzero(G[o])[0][0])
            for sign in (+1, -1):
                keep = np.ones(nsite, dtype=bool)
                cx, cy, cz = x.copy(), y.copy(), z.copy()
                if j == 0:
                    cx = (x + sign) % Lx
                elif j == 1:
                    cy = (y + sign) % Ly
                else:
                    cz = z + sign
                    keep = (cz >= 0) & (cz < Lz)
                sn = (cx + Lx * (cy + Ly * cz))[keep]
                k = int(keep.sum())
                dval = -h * g1[o]
                q = 1.0 if sign < 0 else -1.0
                off = complex(-q * h * G[o, p].imag + 0.0, q * h * G[o, p].real + 0.0)
                rows.append(r[keep]); cols.append(4 * sn + o)
                vals.append(np.full(k, dval, dtype=np.complex128))
                order.append(np.full(k, rank, dtype=np.int64)); rank += 1
                rows.append(r[keep]); cols.append(4 * sn + p)
                vals.append(np.full(k, off, dtype=np.complex128))
                order.append(np.full(k, rank, dtype=np.int64)); rank += 1
    rows = np.concatenate(rows); cols = np.concatenate(cols)
    vals = np.concatenate(vals); order = np.concatenate(order)
    return _merge(rows, cols, vals, order, n, np.complex128)


def topi_slab_clean_spectrum(Lx, Ly, Lz, t=1.0, m=2.0):
    """Eigenvalues of the clean slab from Bloch's theorem in x and y: for each
    (k_x, k_y) the 4 Lz x 4 Lz chain with layer block (m - t cos k_x - t cos k_y)
    Gamma1 + t sin k_x Gamma2 + t sin k_y Gamma3 and layer coupling
    -t (Gamma1 - i Gamma4)/2 from layer z to z+1 (plus Hermitian conjugate)."""
    A = -t * (GAMMA[0] - 1j * GAMMA[3]) / 2.0
    out = []
    for kx in 2 * np.pi * np.arange(Lx) / Lx:
        for ky in 2 * np.pi * np.arange(Ly) / Ly:
            D = ((m - t * np.cos(kx) - t * np.cos(ky)) * GAMMA[0]
                 + t * np.sin(kx) * GAMMA[1] + t * np.sin(ky) * GAMMA[2])
            Hk = np.zeros((4 * Lz, 4 * Lz), dtype=np.complex128)
            for zz in range(Lz):
                Hk[4 * zz:4 * zz + 4, 4 * zz:4 * zz + 4] = D
                if zz + 1 < Lz:
                    Hk[4 * (zz + 1):4 * (zz + 1) + 4, 4 * zz:4 * zz + 4] = A
                    Hk[4 * zz:4 * zz + 4, 4 * (zz + 1):4 * (zz + 1) + 4] = A.conj().T
            out.append(np.linalg.eigvalsh(Hk))
    return np.sort(np.concatenate(out))


def graphene_csr(Lx, Ly, t=1.0, W=0.0, seed=0):
    """CSR (rowptr, col, val float64) of the disordered honeycomb lattice."""
    ncell = Lx * Ly
    n = 2 * ncell
    c = np.arange(ncell, dtype=np.int64)
    i = c % Lx
    j = c // Lx
    V = disorder(seed, n, W)
    rows, cols, vals, order = [], [], [], []

    def cell(ii, jj):
        return (ii % Lx) + Lx * (jj % Ly)

    # sublattice A (0): onsite, B(i,j), B(i-1,j), B(i,j-1)
    rA = 2 * c
    nbA = [cell(i, j), cell(i - 1, j), cell(i, j - 1)]
    # sublattice B (1): onsite, A(i,j), A(i+1,j), A(i,j+1)
    rB = 2 * c + 1
    nbB = [cell(i, j), cell(i + 1, j), cell(i, j + 1)]
    for r, nbs, other in ((rA, nbA, 1), (rB, nbB, 0)):
        rows.append(r); cols.append(r); vals.append(V[r]); order.append(np.zeros(ncell, np.int64))
        for k, nb in enumerate(nbs):
            rows.append(r); cols.append(2 * nb + other)
            vals.append(np.full(ncell, -t)); order.append(np.full(ncell, k + 1, np.int64))
    rows = np.concatenate(rows); cols = np.concatenate(cols)
    vals = np.concatenate(vals); order = np.concatenate(order)
    return _merge(rows, cols, vals, order, n, np.float64)


def flat_dos_eigs(D):
    """lambda_i = -1 + 2 i/(D+1), i = 1..D (Sec. 2.2)."""
    i = np.arange(1, D + 1, dtype=np.float64)
    return -1.0 + 2.0 * i / (D + 1)


def linear_dos_eigs(D):
    """Eigenvalues with rho(lambda) = D |lambda| on [-1, 1] (Sec. 2.4): the flat
    grid s_i mapped through lambda = sgn(s) sqrt|s|, so N_T = D delta^2."""
    s = flat_dos_eigs(D)
    return np.sign(s) * np.sqrt(np.abs(s))


def diagonal_csr(eigs, complex_values=False):
    n = len(eigs)
    rowptr = np.arange(n + 1, dtype=np.int64)
    col = np.arange(n, dtype=np.int32)
    val = np.asarray(eigs, dtype=np.complex128 if complex_values else np.float64)
    return rowptr, col, val


def to_scipy(rowptr, col, val):
    n = len(rowptr) - 1
    return sp.csr_matrix((val, col.astype(np.int64), rowptr), shape=(n, n))


def topi_clean_spectrum(Lx, Ly, Lz, t=1.0, m=1.0):
    """Closed form of the disorder-free insulator: E(k) = +-sqrt((m - t sum cos k)^2
    + t^2 sum sin^2 k), each twice, k_j = 2 pi n_j / L_j (Bloch theorem)."""
    kx = 2 * np.pi * np.arange(Lx) / Lx
    ky = 2 * np.pi * np.arange(Ly) / Ly
    kz = 2 * np.pi * np.arange(Lz) / Lz
    KX, KY, KZ = np.meshgrid(kx, ky, kz, indexing="ij")
    d1 = m - t * (np.cos(KX) + np.cos(KY) + np.cos(KZ))
    s2 = t * t * (np.sin(KX) ** 2 + np.sin(KY) ** 2 + np.sin(KZ) ** 2)
    e = np.sqrt(d1 ** 2 + s2).ravel()
    return np.sort(np.concatenate([e, e, -e, -e]))


def graphene_clean_spectrum(Lx, Ly, t=1.0):
    """Closed form E(k) = +- t |1 + e^{i k1} + e^{i k2}| of the clean honeycomb lattice."""
    k1 = 2 * np.pi * np.arange(Lx) / Lx
    k2 = 2 * np.pi * np.arange(Ly) / Ly
    K1, K2 = np.meshgrid(k1, k2, indexing="ij")
    f = np.abs(1 + np.exp(1j * K1) + np.exp(1j * K2)).ravel()
    return np.sort(np.concatenate([t * f, -t * f]))
