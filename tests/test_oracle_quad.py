"""Pins of the 2D (quadtree) oracle against things other than itself: a
hand-written Morton table, the 2D FFT, exactness when every block is kept at
full rank, an independent sparse assembly of the factors, the adjoint
identity, the dense product at the construction's accuracy, the
complementary low-rank property of the 2D FIO, and planted mistakes that the
exactness pin must catch."""
import numpy as np
import pytest

from bfinputs import complex_normal
from bfinputs.quad import quad_sizes, synthetic_quad_factors
from oracle import quad as Q
from oracle import quad_sparse as QS
from oracle.kernel import rel_err

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def test_morton_order_table():
    """4 x 4 grid: index = sum_b (2 bit_b(p1) + bit_b(p2)) 4^b, written out by
    hand; the first quarter (child 0) is p1, p2 < 2, child 1 has p2 >= 2,
    child 2 has p1 >= 2, child 3 both."""
    expect = [[0, 1, 4, 5],
              [2, 3, 6, 7],
              [8, 9, 12, 13],
              [10, 11, 14, 15]]          # expect[p1][p2]
    p1, p2 = np.meshgrid(np.arange(4), np.arange(4), indexing="ij")
    assert np.array_equal(Q.morton(p1, p2, 2), np.array(expect))
    idx = np.arange(256)
    a, b = Q.demorton(idx, 4)
    assert np.array_equal(Q.morton(a, b, 4), idx)


@pytest.mark.parametrize("n", [4, 16])
def test_dft2_entries_are_the_2d_fft(n):
    """Phi = x.xi: the entry function and the Morton numbering against
    numpy's ifft2 on the grid."""
    g = complex_normal((n * n, 3), seed=1)
    assert rel_err(Q.dense_apply(g, n, "dft2"), Q.dft2_closed_form(g, n)) < 1e-13


@pytest.mark.parametrize("n,L,r", [(4, 2, 4), (8, 2, 16), (16, 2, 64)])
def test_full_rank_factorization_is_exact(n, L, r):
    """With r at least the size of every middle-level block, every block is
    kept whole and the factorization reproduces K to roundoff, forward and
    adjoint (the 2D form of the 1D exactness case)."""
    F = Q.construct(n, L, r, "fio2", seed=2)
    K = Q.entries(np.arange(n * n), np.arange(n * n), n)
    g = complex_normal((n * n, 2), seed=3)
    assert rel_err(Q.bf_apply(F, g), K @ g) < 1e-12
    assert rel_err(Q.bf_adjoint(F, g), K.conj().T @ g) < 1e-12


@pytest.mark.parametrize("L,n0,r", [(2, 1, 2), (2, 4, 5), (4, 1, 3), (4, 4, 6)])
def test_structured_apply_equals_sparse_chain(L, n0, r):
    """Random factors of every ragged shape: the structured apply and adjoint
    equal the product of the factors assembled entry by entry as sparse
    matrices; changing one entry of one block changes both the same way."""
    F = synthetic_quad_factors(L, n0, r, seed=4, dtype=np.complex128)
    g = complex_normal((F.N, 2), seed=5)
    assert rel_err(Q.bf_apply(F, g), QS.chain_apply(F, g)) < 1e-14
    assert rel_err(Q.bf_adjoint(F, g), QS.chain_apply(F, g, adjoint=True)) < 1e-14
    before = Q.bf_apply(F, g)
    F.H[-1][3, 0, 1] += 0.25
    F.G[0][1, 0, 0] -= 0.25
    after = Q.bf_apply(F, g)
    assert rel_err(after, before) > 1e-6
    assert rel_err(after, QS.chain_apply(F, g)) < 1e-14


def test_adjoint_identity_constructed():
    F = Q.construct(16, 4, 8, "fio2", seed=6)
    g = complex_normal((F.N,), seed=7)
    f = complex_normal((F.N,), seed=8)
    Kg = Q.bf_apply(F, g)
    lhs, rhs = np.vdot(f, Kg), np.vdot(Q.bf_adjoint(F, f), g)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(Kg) * np.linalg.norm(f)


def test_fio2_factorization_matches_dense_at_its_accuracy():
    """n = 32 (N = 1024), quadtrees of depth 4 (four points per leaf): the
    factorization error against the dense product is within 10 eps of the
    construction and falls as the rank grows."""
    g = complex_normal((32 * 32, 2), seed=9)
    u = Q.dense_apply(g, 32)
    errs = {}
    for r in (16, 24):
        F = Q.construct(32, 4, r, "fio2", seed=10)
        errs[r] = rel_err(Q.bf_apply(F, g), u)
        assert errs[r] <= 10 * F.meta["eps"]
    assert errs[24] < 2e-2
    assert errs[24] < errs[16] / 3


def test_fio2_middle_blocks_have_slowly_growing_rank():
    """The complementary low-rank property (Sec. 1.1) of the 2D FIO: the
    numerical rank of middle-level blocks at 1e-4 stays near 20 while N grows
    4x (n = 64 -> 128)."""
    ranks = {}
    for n, L in ((64, 6), (128, 7)):
        h = L // 2
        s = Q.block_singular_values(n, L, h, 5, 7)
        ranks[n] = int((s > 1e-4 * s[0]).sum())
    assert ranks[64] <= 24 and ranks[128] <= 26
    assert ranks[128] <= ranks[64] + 4


def test_workload_shape_and_entry_count():
    """The 2D workload's level ranks (24, 24, 16, 4, 1 at levels 4..8) and its
    538,968,064 transfer-block entries (H and G)."""
    s = quad_sizes(8, 1, 24)
    assert s["N"] == 65536 and s["n"] == 256 and s["m"] == 256
    assert s["ranks"] == {4: 24, 5: 24, 6: 16, 7: 4, 8: 1}
    transfer = sum(s["nblocks"] * s["ranks"][lv + 1] * 4 * s["ranks"][lv] for lv in range(4, 8))
    assert 2 * transfer == 538_968_064


def test_exactness_pin_catches_planted_mistakes():
    """Mistakes planted in the oracle's factors, each the effect of a plausible
    slip in the 2D apply (M^h's blocks not transposed, a missing conjugate on
    H^*, the children of a splitting level taken in the wrong order, a leaf
    factor of the wrong leaf): every one breaks the full-rank exactness pin by
    far more than its tolerance, so the pin would catch it."""
    n, L, r = 8, 2, 16
    F = Q.construct(n, L, r, "fio2", seed=21)
    K = Q.entries(np.arange(n * n), np.arange(n * n), n)
    g = complex_normal((n * n,), seed=22)
    ref = K @ g
    assert rel_err(Q.bf_apply(F, g), ref) < 1e-12

    def broken(edit):
        G = Q.QuadFactors(F.L, F.n0, F.r, F.VL.copy(), [a.copy() for a in F.H], F.S.copy(),
                          [a.copy() for a in F.G], F.UL.copy(), dict(F.meta))
        edit(G)
        return rel_err(Q.bf_apply(G, g), ref)

    assert broken(lambda G: G.S.__setitem__(slice(None), F.S.transpose(1, 0, 2))) > 1e-3
    assert broken(lambda G: G.H.__setitem__(0, F.H[0].conj())) > 1e-3
    nb = F.G[0].shape[0]
    order = np.arange(nb).reshape(nb // 4, 4)[:, ::-1].reshape(-1)
    assert broken(lambda G: G.G.__setitem__(0, F.G[0][order])) > 1e-3
    assert broken(lambda G: G.UL.__setitem__(slice(None), F.UL[::-1])) > 1e-3


def test_dft2_factorization_against_the_fft():
    """The 2D DFT (Phi = x.xi) factorized by the 2D construction and applied,
    against numpy's ifft2: within 10 eps of the construction, and improving
    with r (the 2D DFT's blocks have product ranks, so it needs more rank than
    the 1D DFT)."""
    n, L = 16, 4
    g = complex_normal((n * n,), seed=2)
    ref = Q.dft2_closed_form(g, n)
    errs = {}
    for r in (4, 8):
        F = Q.construct(n, L, r, "dft2", seed=1)
        errs[r] = rel_err(Q.bf_apply(F, g), ref)
        assert errs[r] <= 10 * F.meta["eps"]
    assert errs[8] < errs[4] / 5
