"""SELL-C-sigma storage (Sec. 4, Fig. single_socket_perf: SELL-32-1 and SELL-1-1;
format of Kreutzer et al., SIAM J. Sci. Comput. 36 (2014)) - oracle side.

Rows are sorted by length, longest first, inside consecutive windows of sigma
rows (a stable sort: equal lengths keep their original order); the sorted rows
are cut into chunks of C rows; chunk k is padded to its longest row and stored
column-major (entry j of local row l at chunk_ptr[k] + j*C + l).  Padding
entries carry column = the original index of their own row (0 for the slots
past the last row) and value 0.  perm[r] is the original row of sorted row r.
Columns keep the original numbering, so the vectors are not permuted.
"""
import numpy as np


def sell_from_csr(rowptr, col, val, C, sigma):
    n = len(rowptr) - 1
    rowlen = np.diff(rowptr).astype(np.int64)
    perm = np.arange(n, dtype=np.int64)
    if sigma > 1:
        for w0 in range(0, n, sigma):
            w1 = min(w0 + sigma, n)
            order = np.argsort(-rowlen[w0:w1], kind="stable")
            perm[w0:w1] = w0 + order
    nchunks = (n + C - 1) // C
    chunk_len = np.zeros(nchunks, dtype=np.int32)
    for k in range(nchunks):
        rows = perm[k * C:min((k + 1) * C, n)]
        chunk_len[k] = rowlen[rows].max() if len(rows) else 0
    chunk_ptr = np.zeros(nchunks + 1, dtype=np.int64)
    chunk_ptr[1:] = np.cumsum(chunk_len.astype(np.int64) * C)
    total = int(chunk_ptr[-1])
    scol = np.zeros(total, dtype=np.int32)
    sval = np.zeros(total, dtype=val.dtype)
    for k in range(nchunks):
        for l in range(C):
            r = k * C + l
            if r >= n:
                continue
            orig = perm[r]
            b, e = rowptr[orig], rowptr[orig + 1]
            for j in range(chunk_len[k]):
                pos = chunk_ptr[k] + j * C + l
                if j < e - b:
                    scol[pos] = col[b + j]
                    sval[pos] = val[b + j]
                else:
                    scol[pos] = orig
    return dict(n=n, C=C, sigma=sigma, nchunks=nchunks, chunk_ptr=chunk_ptr,
                chunk_len=chunk_len, col=scol, val=sval, perm=perm)


def sell_to_dense_rows(S):
    """Rebuild (rowptr, col, val) in original row order from a SELL structure,
    dropping the padding (used to check the round trip)."""
    n, C = S["n"], S["C"]
    rows = [[] for _ in range(n)]
    for k in range(S["nchunks"]):
        for l in range(C):
            r = k * C + l
            if r >= n:
                continue
            orig = S["perm"][r]
            for j in range(S["chunk_len"][k]):
                pos = S["chunk_ptr"][k] + j * C + l
                rows[orig].append((S["col"][pos], S["val"][pos]))
    return rows
