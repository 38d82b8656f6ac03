"""Order-3 problems with edge ranks above 8 on the GPU, against the FP64 oracle.

The multispectral rank grid of Sec. 5.2 reaches R_{1,2} = 36.  Such shapes run
the chain kernels: M_k and K_k of Prop. 1 as two batched products each, and
column solves with H in shared memory (Cholesky in FP64).  Checked here, all
through the C ABI:

- FP64 path: factors and completed tensor within 1e-10 relative of the oracle
  after one sweep from the same state and after ten sweeps; the rel-change
  and objective of the sweep within 1e-9;
- the mode systems: E_j^T K_k E_j and E_j^T M_k(j,:) equal the oracle's block
  systems A_j^T A_j and A_j^T x_j for every block and column (1e-11);
- mixed path: RSE after 40 sweeps within 1e-3 relative of the oracle's;
- the same result twice, bit for bit (fixed summation orders);
- the limits: ranks up to 64 at order 3, every Q_k <= 4096, ranks above 8
  refused at orders 2 and 4.
"""
import numpy as np
import pytest

import oracle
from paper_2511_16358_gb300 import binding as b
from paper_2511_16358_gb300 import inputs as inp
from tests._cases import make_case, rel_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-10

WIDE = [
    ((24, 20, 10), {(0, 1): 36, (0, 2): 9, (1, 2): 9}),     # the grid's largest point
    ((17, 23, 13), {(0, 1): 12, (0, 2): 3, (1, 2): 10}),    # ragged sizes, mixed ranks
    ((9, 70, 40), {(0, 1): 15, (0, 2): 6, (1, 2): 9}),      # several tiles of every link
    ((40, 9, 70), {(0, 1): 3, (0, 2): 20, (1, 2): 4}),      # wide links (> 16 columns), k = 2 by cost
    ((1, 12, 9), {(0, 1): 10, (0, 2): 2, (1, 2): 3}),       # size-1 mode
    ((5, 6, 3), {(0, 1): 9, (0, 2): 64, (1, 2): 9}),        # the largest rank, Q_k = 576
]


def _ctx(case, precision=b.FP64, max_sweeps=10):
    dt = b.tensor_dtype(precision)
    return b.Completion(case["dims"], case["R"], case["xt"].astype(dt), case["mask"], rho=0.1,
                        max_sweeps=max_sweeps, tol=0.0, precision=precision, init_factors=case["G0"].copy())


@pytest.mark.parametrize("dims,edge", WIDE)
def test_one_sweep_fp64_matches_oracle(dims, edge):
    case = make_case(dims, edge, 0.4, seed=sum(dims) + 7)
    c = _ctx(case)
    st = c.sweep(1)
    G, X = case["G0"].copy(), case["X0"].copy()
    ost = oracle.sweep(dims, case["R"], 0.1, G, X, case["mask"])
    assert rel_err(c.factors(), G) < TOL64
    assert rel_err(c.x(), X) < TOL64
    assert abs(st["rel_change"] - ost["rel_change"]) <= 1e-9 * max(ost["rel_change"], 1e-300)
    assert abs(st["objective"] - ost["objective"]) <= 1e-9 * max(ost["objective"], 1e-300)
    c.close()


@pytest.mark.parametrize("dims,edge", WIDE[:2])
def test_ten_sweeps_fp64_match_oracle(dims, edge):
    case = make_case(dims, edge, 0.3, seed=5)
    c = _ctx(case)
    c.sweep(10)
    G, X = case["G0"].copy(), case["X0"].copy()
    oracle.complete(dims, case["R"], 0.1, G, X, case["mask"], max_sweeps=10)
    assert rel_err(c.factors(), G) < TOL64
    assert rel_err(c.x(), X) < TOL64
    c.close()


@pytest.mark.parametrize("dims,edge", [WIDE[1], WIDE[3]])
def test_mode_systems_match_oracle_block_systems(dims, edge):
    case = make_case(dims, edge, 0.5, seed=11)
    c = _ctx(case)
    N = len(dims)
    R = case["R"]
    F = inp.unpack_factors(case["G0"], dims, R)
    for k in range(N):
        others = [m for m in range(N) if m != k]
        Q = int(np.prod([R[k][m] for m in others]))
        Mk = np.zeros((dims[k], Q))
        Kk = np.zeros((Q, Q))
        b.mode_system(c.ctx, k, Mk, Kk)
        np.testing.assert_allclose(Kk, Kk.T, rtol=1e-12, atol=1e-12 * np.abs(Kk).max())
        for i in others:
            for j in range(dims[k]):
                vecs = [np.eye(R[k][m]) if m == i else F[(k, m)][:, j][:, None] for m in others]
                E = np.kron(vecs[0], vecs[1])
                Ho, bo = oracle.block_system(dims, R, case["G0"], case["X0"], k, i, j)
                assert rel_err(E.T @ Kk @ E, Ho) < 1e-11
                assert rel_err(E.T @ Mk[j], bo) < 1e-11
    c.close()


@pytest.mark.parametrize("dims,edge", [((40, 36, 31), {(0, 1): 15, (0, 2): 6, (1, 2): 6}),
                                       ((32, 30, 12), {(0, 1): 36, (0, 2): 3, (1, 2): 3})])
def test_mixed_precision_rse_within_bound_of_fp64_oracle(dims, edge):
    case = make_case(dims, edge, 0.2, seed=61, kind="minmax01", sigma=0.01)
    n = 40
    c = _ctx(case, precision=b.MIXED, max_sweeps=n)
    c.sweep(n)
    G, X = case["G0"].copy(), case["X0"].copy()
    oracle.complete(dims, case["R"], 0.1, G, X, case["mask"], max_sweeps=n)
    rse_o, _ = oracle.metrics(case["xt"], X, case["mask"])
    rse_g, _ = oracle.metrics(case["xt"], c.x().astype(np.float64), case["mask"])
    assert abs(rse_g - rse_o) <= 1e-3 * rse_o, (rse_g, rse_o)
    c.close()


def test_deterministic_bitwise():
    dims, edge = WIDE[2]
    case = make_case(dims, edge, 0.3, seed=51)
    outs = []
    for _ in range(2):
        c = _ctx(case, precision=b.MIXED)
        c.sweep(5)
        outs.append((c.factors(), c.x()))
        c.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


def test_rank_limits():
    dims = (6, 5, 4)
    xt = np.zeros(dims)
    mask = np.ones(dims, np.uint8)
    for R, ok in [({(0, 1): 64, (0, 2): 64, (1, 2): 1}, True),     # Q_0 = 4096
                  ({(0, 1): 65, (0, 2): 2, (1, 2): 2}, False),
                  ({(0, 1): 64, (0, 2): 65, (1, 2): 1}, False)]:
        rm = inp.rank_matrix(3, R)
        if ok:
            b.Completion(dims, rm, xt, mask, rho=0.1, max_sweeps=1, tol=0.0, precision=b.FP64).close()
        else:
            with pytest.raises(b.IfctnError):
                b.Completion(dims, rm, xt, mask, rho=0.1, max_sweeps=1, tol=0.0, precision=b.FP64)
    with pytest.raises(b.IfctnError):
        b.Completion((4, 3, 5, 2), inp.rank_matrix(4, 9), np.zeros((4, 3, 5, 2)), np.ones((4, 3, 5, 2), np.uint8),
                     rho=0.1, max_sweeps=1, tol=0.0, precision=b.FP64)
