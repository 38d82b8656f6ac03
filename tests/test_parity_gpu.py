"""GPU path vs the FP64 oracle, through the C ABI.

FP64 path: every factor and the completed tensor within 1e-10 relative
(max-abs error over max-abs value) of the oracle after one sweep from the same
state, and after whole runs.  Mixed path (FP32 tensor and contractions, FP64
solves): RSE within 1e-3 relative of the oracle's.
"""

import numpy as np
import pytest

import oracle
from paper_2511_16358_gb300 import binding as b
from paper_2511_16358_gb300 import inputs as inp
from tests._cases import make_case, path, rel_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-10

# "persistent": one cooperative launch per call (the default for tensors that
# stay in L2); "graph": per-stage kernels with the warp-pipelined contraction
# (the default for HBM-sized tensors), forced here on small shapes.
PATHS = ["persistent", "graph"]


def _ctx(case, precision=b.FP64, rho=0.1, max_sweeps=10, tol=0.0):
    dt = b.tensor_dtype(precision)
    c = b.Completion(case["dims"], case["R"], case["xt"].astype(dt), case["mask"], rho=rho,
                     max_sweeps=max_sweeps, tol=tol, precision=precision,
                     init_factors=case["G0"].copy())
    return c


SHAPES = [
    ((7, 9, 5), {(0, 1): 2, (0, 2): 3, (1, 2): 2}),          # N=3 ragged
    ((13, 6, 11), 3),                                       # N=3 odd sizes
    ((5, 7, 4, 6), {(0, 1): 2, (0, 2): 3, (0, 3): 1, (1, 2): 2, (1, 3): 3, (2, 3): 2}),  # N=4 mixed ranks
    ((9, 8), 4),                                            # N=2
    ((4, 3, 5, 8), 1),                                      # rank 1 everywhere
    ((6, 5, 7), 8),                                         # maximum rank
    ((1, 6, 5), 2),                                         # degenerate size-1 mode
    ((6, 5, 1), 2),                                         # size-1 contiguous mode
]


@pytest.mark.parametrize("which", PATHS)
@pytest.mark.parametrize("dims,edge", SHAPES + [
    ((9, 7, 6, 24), {(0, 1): 2, (0, 2): 3, (0, 3): 4, (1, 2): 5, (1, 3): 3, (2, 3): 2}),  # 16-byte rows
    ((5, 4, 70, 36), 3),                                    # row blocks and column chunks
    ((3, 130, 40), {(0, 1): 7, (0, 2): 8, (1, 2): 6}),      # two row blocks, two column chunks
])
def test_one_sweep_fp64_matches_oracle(dims, edge, which):
    case = make_case(dims, edge, 0.4, seed=sum(dims))
    with path(which):
        c = _ctx(case)
    st = c.sweep(1)
    G, X = case["G0"].copy(), case["X0"].copy()
    ost = oracle.sweep(dims, case["R"], 0.1, G, X, case["mask"])
    assert rel_err(c.factors(), G) < TOL64
    assert rel_err(c.x(), X) < TOL64
    assert abs(st["rel_change"] - ost["rel_change"]) <= 1e-9 * max(ost["rel_change"], 1e-300)
    assert abs(st["objective"] - ost["objective"]) <= 1e-9 * max(ost["objective"], 1e-300)
    c.close()


@pytest.mark.parametrize("which", PATHS)
@pytest.mark.parametrize("dims,edge", [
    ((30, 30, 30), 3),
    ((8, 9, 10, 11), 2),
])
def test_whole_run_fp64_matches_oracle(dims, edge, which):
    """Config of the small planted workload: 30^3, R = 3, 30% observed, 50 sweeps."""
    case = make_case(dims, edge, 0.3, seed=5)
    n = 50 if len(dims) == 3 else 20
    with path(which):
        c = _ctx(case, max_sweeps=n)
    c.sweep(n)
    G, X = case["G0"].copy(), case["X0"].copy()
    oracle.complete(dims, case["R"], 0.1, G, X, case["mask"], max_sweeps=n)
    assert rel_err(c.factors(), G) < TOL64
    assert rel_err(c.x(), X) < TOL64
    c.close()


@pytest.mark.parametrize("which", PATHS)
@pytest.mark.parametrize("dims,edge", SHAPES[:3] + [((6, 5, 7, 8), 3)])
def test_mode_systems_match_oracle_block_systems(dims, edge, which):
    """Prop. 1 regrouping on the GPU: H_j = E_j^T K_k E_j and b_j = E_j^T M_k(j,:)
    equal the oracle's A_j^T A_j and A_j^T x_j, for every block (k, i) and column j."""
    case = make_case(dims, edge, 0.5, seed=11)
    with path(which):
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
        for t, i in enumerate(others):
            for j in range(dims[k]):
                vecs = [np.eye(R[k][m]) if m == i else F[(k, m)][:, j][:, None] for m in others]
                E = vecs[0]
                for v in vecs[1:]:
                    E = np.kron(E, v)
                H = E.T @ Kk @ E
                bb = E.T @ Mk[j]
                Ho, bo = oracle.block_system(dims, R, case["G0"], case["X0"], k, i, j)
                assert rel_err(H, Ho) < 1e-11
                assert rel_err(bb, bo) < 1e-11
    c.close()


@pytest.mark.parametrize("precision", [b.FP64, b.MIXED])
def test_reconstruct_matches_oracle(precision):
    dims, edge = (11, 7, 9, 5), {(0, 1): 3, (0, 2): 2, (0, 3): 4, (1, 2): 2, (1, 3): 1, (2, 3): 3}
    case = make_case(dims, edge, 0.5, seed=21)
    c = _ctx(case, precision=precision)
    ref = oracle.reconstruct(dims, case["R"], case["G0"])
    assert rel_err(c.reconstruct(), ref) < (1e-13 if precision == b.FP64 else 2e-6)
    c.close()


def test_observed_entries_bitwise_unchanged_and_x0():
    dims = (10, 9, 8)
    case = make_case(dims, 2, 0.35, seed=31)
    for precision in (b.FP64, b.MIXED):
        c = _ctx(case, precision=precision)
        dt = b.tensor_dtype(precision)
        x0 = c.x()
        obs = case["mask"].astype(bool)
        np.testing.assert_array_equal(x0[obs], case["xt"].astype(dt)[obs])
        np.testing.assert_array_equal(x0[~obs], 0)
        c.sweep(3)
        x3 = c.x()
        np.testing.assert_array_equal(x3[obs], x0[obs])
        c.close()


def test_full_observation_planted_fixed_point():
    dims = (9, 8, 7, 6)
    case = make_case(dims, 2, 1.0, seed=41, kind="raw")
    c = b.Completion(dims, case["R"], case["xt"], case["mask"], rho=0.1, max_sweeps=5, tol=0.0,
                     init_factors=case["Gtrue"].copy())
    st = c.sweep(2)
    assert rel_err(c.factors(), case["Gtrue"]) < 1e-11
    np.testing.assert_array_equal(c.x(), case["xt"])
    assert st["objective"] <= 1e-20 * np.sum(case["xt"] ** 2)
    c.close()


@pytest.mark.parametrize("which", PATHS)
def test_deterministic_bitwise(which):
    dims = (20, 17, 13, 8) if which == "graph" else (20, 17, 13)
    case = make_case(dims, 3, 0.3, seed=51)
    outs = []
    for _ in range(2):
        with path(which):
            c = _ctx(case, precision=b.MIXED)
        c.sweep(5)
        outs.append((c.factors(), c.x()))
        c.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("which,dims", [("persistent", (40, 36, 31)), ("graph", (40, 36, 31)),
                                        ("graph", (12, 16, 15, 24))])
def test_mixed_precision_rse_within_bound_of_fp64_oracle(which, dims):
    case = make_case(dims, 4, 0.2, seed=61, kind="minmax01", sigma=0.01)
    n = 40
    with path(which):
        c = _ctx(case, precision=b.MIXED, max_sweeps=n)
    c.sweep(n)
    G, X = case["G0"].copy(), case["X0"].copy()
    oracle.complete(dims, case["R"], 0.1, G, X, case["mask"], max_sweeps=n)
    rse_o, _ = oracle.metrics(case["xt"], X, case["mask"])
    rse_g, _ = oracle.metrics(case["xt"], c.x().astype(np.float64), case["mask"])
    assert abs(rse_g - rse_o) <= 1e-3 * rse_o, (rse_g, rse_o)
    c.close()


def test_convergence_stop_and_log():
    dims = (12, 11, 10)
    case = make_case(dims, 2, 0.5, seed=71)
    c = _ctx(case, max_sweeps=500, tol=1e-5)
    st = c.complete()
    G, X = case["G0"].copy(), case["X0"].copy()
    log = oracle.complete(dims, case["R"], 0.1, G, X, case["mask"], max_sweeps=500, tol=1e-5)
    assert st["sweeps_done"] == len(log)
    assert st["converged"] == (1 if log[-1]["rel_change"] < 1e-5 else 0)
    glog = b.get_log(c.ctx)
    assert len(glog) == len(log)
    for a, o in zip(glog, log):
        assert abs(a["rel_change"] - o["rel_change"]) <= 1e-8 * o["rel_change"] + 1e-300
    c.close()


def test_metrics_logging_rse_rmse():
    dims = (15, 14, 13)
    case = make_case(dims, 3, 0.3, seed=81, kind="minmax01", sigma=0.01)
    c = _ctx(case, max_sweeps=4)
    b.set_truth(c.ctx, case["xt"], log=True)
    st = c.sweep(4)
    rse, rmse = oracle.metrics(case["xt"], c.x(), case["mask"])
    assert abs(st["rse"] - rse) <= 1e-12 * rse
    assert abs(st["rmse"] - rmse) <= 1e-12 * rmse
    c.close()


def test_checkpoint_resume_is_exact():
    dims = (14, 9, 12)
    case = make_case(dims, 3, 0.4, seed=91)
    c1 = _ctx(case)
    c1.sweep(6)
    ref_G, ref_X = c1.factors(), c1.x()
    c2 = _ctx(case)
    c2.sweep(3)
    G3, X3 = c2.factors(), c2.x()
    c2.close()
    c3 = _ctx(case)
    c3.set_factors(G3)
    c3.set_x(X3)
    c3.sweep(3)
    np.testing.assert_array_equal(c3.factors(), ref_G)
    np.testing.assert_array_equal(c3.x(), ref_X)
    c1.close()
    c3.close()


def test_whole_run_is_one_persistent_launch():
    """A sweep call runs every sweep in one cooperative launch when the grid fits."""
    dims = (32, 28, 24)
    case = make_case(dims, 3, 0.3, seed=101)
    c = _ctx(case, precision=b.MIXED, max_sweeps=20)
    n0 = b.launch_count(c.ctx)
    c.sweep(20)
    assert b.launch_count(c.ctx) - n0 == 1
    c.close()


@pytest.mark.parametrize("cta", ["0", "1"])
@pytest.mark.parametrize("dims,edge", [SHAPES[0], SHAPES[2], ((6, 5, 7), 8), ((9, 7, 6, 24), 3)])
def test_graph_path_both_column_solvers_match_oracle(dims, edge, cta, monkeypatch):
    """The sweep graph's column solves with a warp per column (the default) and
    with a CTA per column (the solve of ranks above 8, selected here): one FP64
    sweep each, within 1e-10 of the oracle."""
    monkeypatch.setenv("IFCTN_CTA_SOLVE", cta)
    case = make_case(dims, edge, 0.4, seed=sum(dims) + 3)
    with path("graph"):
        c = _ctx(case)
    c.sweep(1)
    G, X = case["G0"].copy(), case["X0"].copy()
    oracle.sweep(dims, case["R"], 0.1, G, X, case["mask"])
    assert rel_err(c.factors(), G) < TOL64
    assert rel_err(c.x(), X) < TOL64
    c.close()


@pytest.mark.parametrize("gemm", ["0", "1"])
@pytest.mark.parametrize("dims,edge", [((5, 130, 7, 6), 3), ((6, 9, 5, 4), {(0, 1): 2, (0, 2): 3, (0, 3): 4,
                                                                               (1, 2): 2, (1, 3): 3, (2, 3): 2})])
def test_order4_gram_chain_both_forms_match_oracle_block_systems(dims, edge, gemm, monkeypatch):
    """The order-4 Gram K_k of the sweep graph by one CTA per i_o (the default)
    and by two batched products over i_o (IFCTN_GRAM_GEMM=1): E_j^T K_k E_j
    equals the oracle's A_j^T A_j for every block and column (1e-11)."""
    monkeypatch.setenv("IFCTN_GRAM_GEMM", gemm)
    case = make_case(dims, edge, 0.5, seed=13)
    with path("graph"):
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
        for i in others:
            for j in range(0, dims[k], max(1, dims[k] // 7)):
                vecs = [np.eye(R[k][m]) if m == i else F[(k, m)][:, j][:, None] for m in others]
                E = vecs[0]
                for v in vecs[1:]:
                    E = np.kron(E, v)
                Ho, _ = oracle.block_system(dims, R, case["G0"], case["X0"], k, i, j)
                assert rel_err(E.T @ Kk @ E, Ho) < 1e-11
    c.close()
