"""Tiny independent GF(2) helpers for the tests (numpy, written separately from
the oracle so that pins do not re-call the code they check)."""
import numpy as np


def rref(M):
    A = (np.asarray(M) & 1).astype(np.uint8).copy()
    rows, cols = A.shape
    piv = []
    r = 0
    for c in range(cols):
        if r >= rows:
            break
        nz = np.nonzero(A[r:, c])[0]
        if len(nz) == 0:
            continue
        p = r + nz[0]
        if p != r:
            A[[r, p]] = A[[p, r]]
        hit = np.nonzero(A[:, c])[0]
        hit = hit[hit != r]
        A[hit] ^= A[r]
        piv.append(c)
        r += 1
    return A[:r], piv


def rank(M):
    return len(rref(M)[1])


def nullspace(M):
    """Basis (rows) of {x : M x = 0}."""
    R, piv = rref(M)
    n = M.shape[1]
    free = [c for c in range(n) if c not in set(piv)]
    out = []
    for f in free:
        v = np.zeros(n, np.uint8)
        v[f] = 1
        for i, pc in enumerate(piv):
            if R[i, f]:
                v[pc] = 1
        out.append(v)
    return np.array(out, np.uint8).reshape(len(out), n)
