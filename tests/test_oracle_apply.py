"""Pins of the oracle apply/adjoint (Eq. Kfactors) against the brute-force
sparse assembly of the paper's block matrices, the C loops and the adjoint
identity; and of the index structure against the paper's N = 64 figures."""
import os

import numpy as np
import pytest

from bfinputs import complex_normal, synthetic_factors
from oracle import apply as A
from oracle import capply as CA
from oracle import kernel as K
from oracle import sparse as SP

SHAPES = [(0, 5, 3), (2, 2, 3), (2, 1, 4), (4, 1, 2), (4, 3, 5), (6, 1, 1), (6, 2, 3), (8, 1, 2)]


@pytest.mark.parametrize("L,n0,r", SHAPES)
def test_apply_matches_sparse_chain_and_c(L, n0, r):
    F = synthetic_factors(L, n0, r, seed=L + 10 * r, dtype=np.complex128)
    g = complex_normal((F.N, 3), seed=4)
    ref = SP.chain_apply(F, g)
    assert K.rel_err(A.bf_apply(F, g), ref) < 1e-13
    assert K.rel_err(CA.bf_apply_c(F, g), ref) < 1e-13
    refa = SP.chain_apply(F, g, adjoint=True)
    assert K.rel_err(A.bf_adjoint(F, g), refa) < 1e-13
    assert K.rel_err(CA.bf_adjoint_c(F, g), refa) < 1e-13


@pytest.mark.parametrize("L,n0,r", [(4, 2, 3), (6, 1, 2)])
def test_adjoint_identity(L, n0, r):
    """<K g, f> = <g, K^* f> for the oracle apply of any factors."""
    F = synthetic_factors(L, n0, r, seed=3, dtype=np.complex128)
    g = complex_normal((F.N,), seed=5)
    f = complex_normal((F.N,), seed=6)
    lhs = np.vdot(f, A.bf_apply(F, g))
    rhs = np.vdot(A.bf_adjoint(F, f), g)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(A.bf_apply(F, g)) * np.linalg.norm(f)
    D = SP.dense_product(F)
    assert np.allclose(D.conj().T @ f, A.bf_adjoint(F, f), atol=1e-12)


def test_vector_and_matrix_inputs_agree():
    F = synthetic_factors(4, 2, 3, seed=1, dtype=np.complex128)
    g = complex_normal((F.N, 4), seed=2)
    cols = np.stack([A.bf_apply(F, g[:, c]) for c in range(4)], axis=1)
    assert np.allclose(cols, A.bf_apply(F, g), atol=1e-14)


def test_planted_mistakes_are_caught(monkeypatch):
    """Plausible mistakes planted in the oracle apply -- the conjugation of
    (V^L)^* and (H^l)^* dropped, or S^h_{i,j} read as S^h_{j,i} -- are caught
    by the sparse cross-check (complex factors, S not symmetric)."""
    F = synthetic_factors(4, 2, 3, seed=2, dtype=np.complex128)
    g = complex_normal((F.N,), seed=3)
    ref = SP.chain_apply(F, g)
    assert K.rel_err(A.bf_apply(F, g), ref) < 1e-13
    Fb = type(F)(F.L, F.n0, F.r, F.VL, F.H, F.S.transpose(1, 0, 2).copy(), F.G, F.UL)
    assert K.rel_err(A.bf_apply(Fb, g), ref) > 1e-3
    with monkeypatch.context() as mp:
        mp.setattr(A.np, "conj", lambda x: x)
        assert K.rel_err(A.bf_apply(F, g), ref) > 1e-3


def _read_patterns(path):
    mats, cur = {}, None
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("matrix"):
            _, name, nr, nc = line.split()[:4]
            cur = name
            mats[name] = (int(nr), int(nc), set())
        else:
            row, cols = line.split(":")
            for c in cols.split():
                mats[cur][2].add((int(row), int(c)))
    return mats


def _pattern(M):
    M = M.tocoo()
    return {(int(a), int(b)) for a, b, v in zip(M.row, M.col, M.data) if v != 0}


def test_block_structure_matches_paper_figures(repo_root):
    """Sparsity of U^3, M^3, (V^3)^*, U^4, G^3, U^5, G^4, (H^3)^*, (H^4)^*, (V^5)^*
    for N = 64, L = 6, r = 1 (Figs. compression-1D, -1D2, -1D3), bit-exact
    against the brute-force assembly of the block-matrix definitions."""
    mats = _read_patterns(os.path.join(repo_root, "tests", "golden", "fig_n64_patterns.txt"))
    N, L, r = 64, 6, 1
    ones_t = np.ones((1 << L, r, 2 * r), dtype=complex)

    def basis(level):
        return SP.level_basis_matrix(np.ones((1 << level, 1 << (L - level), N >> level, r)))

    built = {
        "U3": basis(3), "U4": basis(4), "U5": basis(5),
        "V3h": basis(3).conj().T, "V5h": basis(5).conj().T,
        "M3": SP.middle_matrix(np.ones((8, 8, r)), r),
        "G3": SP.transfer_matrix(ones_t, 3, L, r), "G4": SP.transfer_matrix(ones_t, 4, L, r),
        "H3h": SP.transfer_matrix(ones_t, 3, L, r).conj().T,
        "H4h": SP.transfer_matrix(ones_t, 4, L, r).conj().T,
    }
    assert set(built) == set(mats)
    for name, M in built.items():
        nr, nc, nz = mats[name]
        assert M.shape == (nr, nc), name
        assert _pattern(M) == nz, name
