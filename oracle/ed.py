"""Exact diagonalisation from operator-term lists (pins only).

Test infrastructure (see the package header). The Hamiltonian is assembled
as a sum of Kronecker products of the local matrices of each term, with
identities elsewhere -- the textbook definition of a many-body operator,
independent of the MPO construction. Eigenvalues come from
``numpy.linalg.eigh`` (dense) or ``scipy.sparse.linalg.eigsh`` (sparse,
restricted to one conserved-charge sector).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _term_sparse(N, d, coef, ops):
    fac = dict(ops)
    mat = sp.identity(1, format="csr")
    for i in range(N):
        m = sp.csr_matrix(fac[i]) if i in fac else sp.identity(d, format="csr")
        mat = sp.kron(mat, m, format="csr")
    return coef * mat


def hamiltonian_sparse(N, d, terms):
    """Sparse full Hamiltonian; site 0 is the slowest Kronecker factor."""
    H = sp.csr_matrix((d ** N, d ** N))
    for coef, ops in terms:
        H = H + _term_sparse(N, d, coef, ops)
    return H.tocsr()


def _require_symmetric(H):
    """A real Hamiltonian is a symmetric matrix. The eigensolvers below read
    one triangle only, so a term list that breaks the symmetry (a missing or
    mis-signed Hermitian conjugate) would pass unnoticed: refuse it."""
    D = abs(H - H.T)
    big = abs(H).max() if (H.nnz if sp.issparse(H) else H.size) else 0.0
    if D.max() > 1e-12 * max(1.0, float(big)):
        raise ValueError("the Hamiltonian built from these terms is not symmetric")


def hamiltonian_dense(N, d, terms):
    H = hamiltonian_sparse(N, d, terms).toarray()
    _require_symmetric(H)
    return H


def basis_charges(N, site_qn):
    """Total charge of every product basis state (same ordering as above)."""
    d = len(site_qn)
    q = np.asarray(site_qn)                      # (d, nq)
    tot = np.zeros((1, q.shape[1]), dtype=np.int64)
    for _ in range(N):
        tot = (tot[:, None, :] + q[None, :, :]).reshape(-1, q.shape[1])
    return tot


def ground_energy(N, d, terms, site_qn=None, sector=None, k=1):
    """Lowest eigenvalue(s), optionally inside one total-charge sector."""
    H = hamiltonian_sparse(N, d, terms)
    if sector is not None:
        ch = basis_charges(N, site_qn)
        sel = np.nonzero(np.all(ch == np.asarray(sector)[None, :], axis=1))[0]
        H = H[sel][:, sel]
    _require_symmetric(H)
    n = H.shape[0]
    if n <= 4096:
        w = np.linalg.eigh(H.toarray())[0]
        return w[:k] if k > 1 else float(w[0])
    w = spla.eigsh(H, k=max(k, 1), which="SA", tol=1e-13, maxiter=20000)[0]
    w = np.sort(w)
    return w[:k] if k > 1 else float(w[0])
