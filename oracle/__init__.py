"""FP64 CPU oracle for the butterfly factorization (Li, Yang, Martin, Ho, Ying,
"Butterfly Factorization", arXiv 1502.01379).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA path (``paper_1502_01379_gb300``); the two
meet only through the seeded input generators in ``bfinputs``, which hold none
of the method's arithmetic.

Modules (each function cites the passage of the paper it follows):

* ``kernel``   -- the entry function K(x, xi) = exp(2 pi i Phi(x, xi)) of the
                  Fourier matrix (Sec. 1.1) and of Example 1 (Sec. 4), with the
                  phase reduced modulo 1 exactly; the dense product u = K g.
* ``lowrank``  -- the rank-r SVD forms (Eqs. lowrankSVD/2/3) and the
                  randomized-sampling low-rank approximation (Sec. 2.2).
* ``construct``-- the middle-level factorization (Sec. 3.1, Eq. KeqUMV) and
                  the recursive factorization of U^h and V^h (Sec. 3.2),
                  in the memory-saving row-node-at-a-time order (Sec. 3.3).
* ``construct_mv`` -- the construction when only K g and K^* g are available
                  (Sec. 3.1, first case): randomized SVDs of all middle blocks
                  from 2 m (r + p) products (Sec. 2.1), then Sec. 3.2; and the
                  composition K F K of Example 3 (Sec. 4).
* ``apply``    -- the apply u = U^L G^{L-1}...G^h M^h (H^h)^*...(H^{L-1})^* (V^L)^* g
                  of Eq. (Kfactors) and its adjoint, one factor at a time.
* ``grad``     -- reverse mode through the same chain: the gradient of a real
                  loss with respect to the input and to every factor block
                  (differentiation of the apply; PyTorch's complex convention).
* ``sparse``   -- an independent brute-force path: every factor assembled as
                  an explicit sparse matrix from the block-matrix displays of
                  Sec. 3, and the chain multiplied out.
* ``quad``     -- the 2D carry-over on quadtrees (Sec. 1.2 notes it exists;
                  the readings it takes are in its docstring): Morton order,
                  a 2D FIO and the 2D DFT, construction with four children per
                  node, apply and adjoint.
* ``quad_sparse``-- the 2D factors assembled entry by entry as sparse
                  matrices (independent of ``quad``'s reshapes).
* ``capply``   -- ctypes binding of ``capply.c``: the same apply/adjoint as
                  plain C loops in FP64 (OpenMP over blocks), used for the
                  timed CPU baseline and for full-size parity.

Where the paper is silent or ambiguous, the reading taken is stated in the
docstring of the function that depends on it.
"""
