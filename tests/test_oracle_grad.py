"""Pins of the oracle gradient (reverse mode through Eq. Kfactors) against
what the mathematics fixes, none of which reuses its code:

* brute force: the chain of explicit sparse factor matrices (the independent
  assembly of the paper's block matrices in ``oracle.sparse``), the dense
  gradient of every factor matrix, mapped back to the parameters through a
  second assembly with unique integer IDs as block values;
* the input gradient is the adjoint apply K^* ubar (``oracle.apply``);
* homogeneity: the chain is linear in each factor, so for every factor F,
  Re <Fbar, F> = Re <ubar, u>;
* central finite differences of L = ||K g - y||^2, which is quadratic in
  every single factor entry, so the difference quotient is exact up to
  rounding (step 1e-3 in FP64, a sample of entries of every factor);
* planted mistakes in a gradient (a conjugation, a transposition, a swapped
  half) are caught by the brute force."""
import numpy as np
import pytest

from bfinputs import complex_normal, synthetic_factors
from oracle import apply as A
from oracle import grad as GR
from oracle import kernel as K
from oracle import sparse as SP

SHAPES = [(0, 3, 2), (2, 2, 3), (4, 1, 2), (4, 2, 3), (6, 1, 2)]


def _param_arrays(F):
    """(name, array) of every parameter, in a fixed order."""
    out = [("VL", np.asarray(F.VL))]
    out += [(f"H{t}", np.asarray(F.H[t])) for t in range(F.h)]
    out += [("S", np.asarray(F.S))]
    out += [(f"G{t}", np.asarray(F.G[t])) for t in range(F.h)]
    out += [("UL", np.asarray(F.UL))]
    return out


def _brute_force_grads(F, g, ubar):
    """Parameter gradients from the dense gradients of the sparse factor chain."""
    mats = [M.toarray() for M in SP.factor_list(F)]
    nf = len(mats)
    y = [None] * (nf + 1)
    y[nf] = np.asarray(g, dtype=np.complex128)
    for q in range(nf - 1, -1, -1):
        y[q] = mats[q] @ y[q + 1]
    delta = np.asarray(ubar, dtype=np.complex128)
    dense_grad = [None] * nf
    for q in range(nf):
        dense_grad[q] = delta @ y[q + 1].conj().T
        delta = mats[q].conj().T @ delta
    gbar = delta
    # the same factor list with unique IDs (1-based) as entries of each parameter array
    L, r, h = F.L, F.r, F.h
    ids = {}
    for name, arr in _param_arrays(F):
        ids[name] = np.arange(1, arr.size + 1, dtype=np.float64).reshape(arr.shape)
    id_mats, conj_factor, names = [], [], []
    id_mats.append(SP.leaf_matrix(ids["UL"].astype(np.complex128), F.n0, r)); conj_factor.append(False); names.append("UL")
    for l in range(L - 1, h - 1, -1):
        id_mats.append(SP.transfer_matrix(ids[f"G{l - h}"].astype(np.complex128), l, L, r))
        conj_factor.append(False); names.append(f"G{l - h}")
    id_mats.append(SP.middle_matrix(ids["S"], r)); conj_factor.append(False); names.append("S")
    for l in range(h, L):
        id_mats.append(SP.transfer_matrix(ids[f"H{l - h}"].astype(np.complex128), l, L, r).conj().T.tocsr())
        conj_factor.append(True); names.append(f"H{l - h}")
    id_mats.append(SP.leaf_matrix(ids["VL"].astype(np.complex128), F.n0, r).conj().T.tocsr())
    conj_factor.append(True); names.append("VL")
    grads = {name: np.zeros(arr.shape, dtype=np.complex128) for name, arr in _param_arrays(F)}
    for q in range(nf):
        M = id_mats[q].tocoo()
        for row, col, v in zip(M.row, M.col, M.data):
            idx = int(round(v.real)) - 1
            gv = dense_grad[q][row, col]
            grads[names[q]].flat[idx] += np.conj(gv) if conj_factor[q] else gv
    grads["S"] = grads["S"].real
    return gbar, grads


def _as_dict(grads):
    return {name: arr for name, arr in _param_arrays(grads)}


@pytest.mark.parametrize("L,n0,r", SHAPES)
def test_gradient_matches_sparse_chain(L, n0, r):
    F = synthetic_factors(L, n0, r, seed=40 + L + r, dtype=np.complex128)
    g = complex_normal((F.N, 2), seed=1)
    ubar = complex_normal((F.N, 2), seed=2)
    u, gbar, grads = GR.bf_apply_and_grad(F, g, ubar)
    assert K.rel_err(u, A.bf_apply(F, g)) < 1e-13
    bgbar, bgrads = _brute_force_grads(F, g, ubar)
    assert K.rel_err(gbar, bgbar) < 1e-12
    for name, arr in _as_dict(grads).items():
        assert K.rel_err(arr, bgrads[name]) < 1e-12, name


@pytest.mark.parametrize("L,n0,r", [(4, 2, 3), (8, 2, 3)])
def test_input_gradient_is_adjoint_apply(L, n0, r):
    F = synthetic_factors(L, n0, r, seed=7, dtype=np.complex128)
    g = complex_normal((F.N, 3), seed=3)
    ubar = complex_normal((F.N, 3), seed=4)
    _, gbar, _ = GR.bf_apply_and_grad(F, g, ubar)
    assert K.rel_err(gbar, A.bf_adjoint(F, ubar)) < 1e-13


@pytest.mark.parametrize("L,n0,r", [(4, 2, 3), (8, 4, 4)])
def test_homogeneity_of_every_factor(L, n0, r):
    """u is linear in each factor F, so d/dt L(u(tF)) at t = 1 equals both
    Re <Fbar, F> and Re <ubar, u>."""
    F = synthetic_factors(L, n0, r, seed=9, dtype=np.complex128)
    g = complex_normal((F.N, 2), seed=5)
    ubar = complex_normal((F.N, 2), seed=6)
    u, _, grads = GR.bf_apply_and_grad(F, g, ubar)
    ref = np.vdot(ubar, u).real
    P, Gd = _as_dict(F), _as_dict(grads)
    for name in P:
        val = np.vdot(Gd[name], P[name]).real
        assert abs(val - ref) <= 1e-11 * abs(ref), name


def test_central_finite_differences():
    """L = ||K g - y||^2 is quadratic in each factor entry: the central
    difference with step 1e-3 is exact up to FP64 rounding (sampled entries
    of every factor, real and imaginary directions)."""
    F = synthetic_factors(6, 2, 3, seed=11, dtype=np.complex128)
    g = complex_normal((F.N, 2), seed=7)
    y = complex_normal((F.N, 2), seed=8)
    _, _, _, grads = GR.loss_and_grad(F, g, y)
    Gd = _as_dict(grads)
    rng = np.random.default_rng(0)
    step = 1e-3

    def loss(Fp):
        res = A.bf_apply(Fp, g) - y
        return np.vdot(res, res).real

    for name, arr in _param_arrays(F):
        for flat in rng.choice(arr.size, size=4, replace=False):
            dirs = [1.0] if name == "S" else [1.0, 1j]
            for d in dirs:
                vals = []
                for sgn in (1.0, -1.0):
                    Fp = type(F)(F.L, F.n0, F.r, F.VL.copy(), [a.copy() for a in F.H], F.S.copy(),
                                 [a.copy() for a in F.G], F.UL.copy())
                    target = dict(_param_arrays(Fp))[name]
                    target.flat[flat] += sgn * step * d
                    vals.append(loss(Fp))
                fd = (vals[0] - vals[1]) / (2 * step)
                gv = Gd[name].flat[flat]
                comp = gv.real if d == 1.0 else gv.imag
                assert abs(fd - comp) <= 1e-7 * (1 + abs(comp)), (name, flat, d)


def test_planted_mistakes_are_caught():
    F = synthetic_factors(4, 2, 3, seed=13, dtype=np.complex128)
    g = complex_normal((F.N, 2), seed=9)
    ubar = complex_normal((F.N, 2), seed=10)
    _, _, grads = GR.bf_apply_and_grad(F, g, ubar)
    _, bgrads = _brute_force_grads(F, g, ubar)
    Gd = _as_dict(grads)
    wrong = {
        "H0": np.conj(Gd["H0"]),                                     # a conjugation dropped
        "G1": Gd["G1"][:, :, ::-1].copy(),                           # columns reversed
        "S": Gd["S"].transpose(1, 0, 2).copy(),                      # S_{i,j} read as S_{j,i}
        "VL": np.roll(Gd["VL"], 1, axis=0),                          # blocks shifted by one leaf
    }
    for name, arr in wrong.items():
        assert K.rel_err(arr, bgrads[name]) > 1e-3, name
