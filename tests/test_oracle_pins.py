"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle (oracle/ifctn_oracle.c) against an independent
formulation: brute-force sums over every rank tuple (eq. iFCTN), the FCTN
contraction of cherry cores built by Def. 1 (eq. FCTN), the explicit
sub-network matrix of Prop. 1, transposition invariance (Prop. 3), printed
numbers (Tables 5 and 6), textbook special cases (rank-1 CP, N=2 proximal ALS),
explicit dense least-squares systems for the block updates (eq. updateG),
the monotone decrease of Lemma 2 and the planted fixed point.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2511_16358_gb300 import inputs as inp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _problem(dims, edge, seed, dist="normal"):
    N = len(dims)
    R = inp.rank_matrix(N, edge)
    G = inp.gaussian_factors(dims, R, seed) if dist == "normal" else inp.uniform_factors(dims, R, seed)
    return R, G


def _bruteforce_ifctn(dims, R, G):
    """eq. (iFCTN) literally: for every entry, sum over every tuple of rank
    indices r_{k,l} (k<l) of the product of all N(N-1) cherry-factor entries."""
    N = len(dims)
    F = inp.unpack_factors(G, dims, R)
    pairs = [(k, l) for k in range(N) for l in range(k + 1, N)]
    ranges = [range(int(R[k][l])) for k, l in pairs]
    out = np.zeros(dims)
    for idx in itertools.product(*[range(d) for d in dims]):
        tot = 0.0
        for rt in itertools.product(*ranges):
            r = {}
            for (k, l), rv in zip(pairs, rt):
                r[(k, l)] = r[(l, k)] = rv
            prod = 1.0
            for k in range(N):
                for l in range(N):
                    if l != k:
                        prod *= F[(k, l)][r[(k, l)], idx[k]]
            tot += prod
        out[idx] = tot
    return out


def _khatri_rao(A, B):
    """Column-wise Kronecker product of Sec. 2.1: c_{(i-1)n+j,l} = a_{il} b_{jl}."""
    m, r = A.shape
    n, r2 = B.shape
    assert r == r2
    return (A[:, None, :] * B[None, :, :]).reshape(m * n, r)


def _fold_littleendian(M, shape, k):
    """Inverse of the mode-k unfolding of Sec. 2.1 (first remaining index fastest)."""
    rest = [shape[m] for m in range(len(shape)) if m != k]
    T = M.reshape([shape[k]] + rest, order="F")
    return np.moveaxis(T, 0, k)


def _unfold_littleendian(T, k):
    return np.moveaxis(T, k, 0).reshape(T.shape[k], -1, order="F")


def _cherry_core(dims, R, F, k):
    """Def. 1: core whose mode-k unfolding is (M_N kr ... kr M_{k+1} kr M_{k-1} kr ... kr M_1)^T
    with M_m = G_{k,m}; modes (R_{1,k},...,I_k,...,R_{k,N})."""
    N = len(dims)
    order = [m for m in range(N - 1, -1, -1) if m != k]
    # Def. 1 writes M_m in R^{R_m x I_k}; the KR product of Sec. 2.1 pairs the
    # columns (index i_k), so the product's row index runs over the rank tuple.
    C = F[(k, order[0])]
    for m in order[1:]:
        C = _khatri_rao(C, F[(k, m)])  # rows: rank tuple, first listed factor slowest
    # C is (prod R) x I_k = (G_(k))^T
    shape = [int(R[k][m]) if m != k else int(dims[k]) for m in range(N)]
    return _fold_littleendian(C.T, shape, k)


def _fctn_contract(dims, cores):
    """eq. (FCTN): sum over every rank index of the product of the N cores."""
    N = len(dims)
    letters = iter("abcdefghijklmnopqrstuvwxyz")
    pair_letter = {}
    for k in range(N):
        for l in range(k + 1, N):
            pair_letter[(k, l)] = pair_letter[(l, k)] = next(letters)
    idx_letter = [next(letters) for _ in range(N)]
    subs = []
    for k in range(N):
        subs.append("".join(idx_letter[k] if m == k else pair_letter[(k, m)] for m in range(N)))
    return np.einsum(",".join(subs) + "->" + "".join(idx_letter), *cores)


# ---------------------------------------------------------------------------
# reconstruction, eq. (iFCTN)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,edge,seed", [
    ((3, 4, 2), {(0, 1): 2, (0, 2): 3, (1, 2): 1}, 11),
    ((2, 3, 2, 3), {(0, 1): 2, (0, 2): 1, (0, 3): 2, (1, 2): 2, (1, 3): 1, (2, 3): 2}, 12),
    ((4, 3), {(0, 1): 3}, 13),
])
def test_reconstruct_matches_bruteforce_rank_sum(dims, edge, seed):
    R, G = _problem(dims, edge, seed)
    ref = _bruteforce_ifctn(dims, R, G)
    got = oracle.reconstruct(dims, R, G)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("dims,edge,seed", [
    ((3, 4, 2), {(0, 1): 2, (0, 2): 3, (1, 2): 2}, 21),
    ((2, 3, 4, 2), {(0, 1): 2, (0, 2): 3, (0, 3): 1, (1, 2): 2, (1, 3): 3, (2, 3): 2}, 22),
])
def test_reconstruct_equals_fctn_of_cherry_cores(dims, edge, seed):
    """Def. 1 cores (KR-structured, little-endian unfolding) contracted by eq. (FCTN)."""
    R, G = _problem(dims, edge, seed)
    F = inp.unpack_factors(G, dims, R)
    cores = [_cherry_core(dims, R, F, k) for k in range(len(dims))]
    # the entry of core k at rank tuple r and index i_k is prod_m G_{k,m}(r_m, i_k)
    k = 1
    rr = [0] * len(dims)
    rr[k] = 1
    expect = np.prod([F[(k, m)][0, 1] for m in range(len(dims)) if m != k])
    assert np.isclose(cores[k][tuple(rr)], expect)
    ref = _fctn_contract(dims, cores)
    got = oracle.reconstruct(dims, R, G)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_three_way_remark_formula():
    """The N = 3 remark of Sec. 3: explicit triple sum over r12, r13, r23."""
    dims = (4, 3, 5)
    R, G = _problem(dims, {(0, 1): 3, (0, 2): 2, (1, 2): 4}, 31)
    F = inp.unpack_factors(G, dims, R)
    ref = np.einsum("ai,bi,aj,cj,bk,ck->ijk", F[(0, 1)], F[(0, 2)], F[(1, 0)], F[(1, 2)],
                    F[(2, 0)], F[(2, 1)])
    np.testing.assert_allclose(oracle.reconstruct(dims, R, G), ref, rtol=1e-13, atol=1e-14)


def _cherry_tensor(mats, k, Ik):
    """Def. 1 written out entry by entry: a mode-k cherry tensor with cherry
    factors mats[i] (P_i x I_k, i != k) has entry prod_{i != k} mats[i](p_i, i_k)."""
    N = len(mats)
    shape = [Ik if i == k else mats[i].shape[0] for i in range(N)]
    T = np.zeros(shape)
    for idx in itertools.product(*[range(d) for d in shape]):
        T[idx] = np.prod([mats[i][idx[i], idx[k]] for i in range(N) if i != k])
    return T


def _cherry_product(A, k, B, t, alpha, beta):
    """Def. 3 entry by entry (brute force): A = CT_k({A_i}), B = CT_t({B_j});
    the result has the modes of A without alpha, then those of B without beta,
    and entry prod_{i != k, alpha} A_i(., i_k) * prod_{j != t, beta} B_j(., j_t)
    * (A_alpha^T B_beta)(i_k, j_t)."""
    N, M = len(A), len(B)
    Ik = next(A[i].shape[1] for i in range(N) if i != k)
    Jt = next(B[j].shape[1] for j in range(M) if j != t)
    nA = [i for i in range(N) if i != alpha]
    mB = [j for j in range(M) if j != beta]
    dimA = [Ik if i == k else A[i].shape[0] for i in nA]
    dimB = [Jt if j == t else B[j].shape[0] for j in mB]
    AB = A[alpha].T @ B[beta]
    C = np.zeros(dimA + dimB)
    for ia in itertools.product(*[range(d) for d in dimA]):
        a = dict(zip(nA, ia))
        for jb in itertools.product(*[range(d) for d in dimB]):
            b = dict(zip(mB, jb))
            v = AB[a[k], b[t]]
            for i in nA:
                if i != k:
                    v *= A[i][a[i], a[k]]
            for j in mB:
                if j != t:
                    v *= B[j][b[j], b[t]]
            C[ia + jb] = v
    return C


def test_cherry_product_is_the_contraction_of_the_shared_mode():
    """Def. 3: the cherry product equals summing the product of the two cherry
    tensors over the connected mode (alpha of A, beta of B)."""
    rng = np.random.default_rng(5)
    Ik, Jt = 3, 4
    A = [rng.standard_normal((2, Ik)), None, rng.standard_normal((3, Ik)), rng.standard_normal((2, Ik))]
    B = [rng.standard_normal((3, Jt)), rng.standard_normal((2, Jt)), None]
    k, t, alpha, beta = 1, 2, 2, 0
    TA = _cherry_tensor(A, k, Ik)
    TB = _cherry_tensor(B, t, Jt)
    ref = np.tensordot(TA, TB, axes=([alpha], [beta]))
    np.testing.assert_allclose(_cherry_product(A, k, B, t, alpha, beta), ref, rtol=1e-13, atol=1e-14)


def test_cherry_product_remark_forms():
    """The N = M = 3 remark after Def. 3: a mode-2 cherry tensor (P x I x R) and a
    mode-3 cherry tensor (Q x R x J) give C(p,i,q,j) = A_1(p,i) B_1(q,j) (A_3^T B_2)_{ij};
    matricised, C = diag(vec(A_3^T B_2)) (B_1 kron A_1)^T with rows (i,j), i fastest,
    and columns (p,q), p fastest (the printed column size R_1 R_3 is read as P Q)."""
    rng = np.random.default_rng(6)
    P, I, R, Q, J = 2, 3, 4, 3, 2
    A1, A3 = rng.standard_normal((P, I)), rng.standard_normal((R, I))
    B1, B2 = rng.standard_normal((Q, J)), rng.standard_normal((R, J))
    C = _cherry_product([A1, None, A3], 1, [B1, B2, None], 2, 2, 1)
    assert C.shape == (P, I, Q, J)
    np.testing.assert_allclose(C, np.einsum("pi,qj,ij->piqj", A1, B1, A3.T @ B2), rtol=1e-13, atol=1e-14)
    Cmat = np.diag((A3.T @ B2).reshape(-1, order="F")) @ np.kron(B1, A1).T
    ref = np.transpose(C, (1, 3, 0, 2)).reshape(I * J, P * Q, order="F")
    np.testing.assert_allclose(Cmat, ref, rtol=1e-13, atol=1e-14)


def test_cherry_products_pack_the_subnetwork_and_rebuild_the_tensor():
    """Packing by cherry products (Sec. 3): G_1 * G_2 over r_{1,2} is the
    sub-network of the remaining cherries (its unfolding is Z_3 of Prop. 1),
    and contracting it with G_3 over r_{1,3}, r_{2,3} gives iFCTN(G)."""
    dims = (3, 4, 2)
    R, G = _problem(dims, {(0, 1): 2, (0, 2): 3, (1, 2): 2}, 81)
    F = inp.unpack_factors(G, dims, R)
    c = [[F[(k, m)] if m != k else None for m in range(3)] for k in range(3)]
    C12 = _cherry_product(c[0], 0, c[1], 1, 1, 0)            # modes (i1, r13, i2, r23)
    assert C12.shape == (dims[0], R[0, 2], dims[1], R[1, 2])
    T3 = _cherry_tensor(c[2], 2, dims[2])                      # modes (r13, r23, i3)
    X = np.einsum("asbt,sti->abi", C12, T3)
    np.testing.assert_allclose(X, oracle.reconstruct(dims, R, G), rtol=1e-12, atol=1e-13)
    # rows (i1, i2) with i1 fastest, columns (r13, r23) with r23 slowest: Z_3
    Z3 = np.transpose(C12, (0, 2, 1, 3)).reshape(dims[0] * dims[1], -1, order="F")
    np.testing.assert_allclose(Z3, _prop1_Z(dims, R, F, 2), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_prop1_subnetwork_unfolding(k):
    """Prop. 1: (X_(k))^T = Z_k (G_(k))^T, Z_k = diag(vec S_k) (kron_{i=N..1, i!=k} G_{i,k}^T),
    S_k the broadcast product of G_{i,j}^T G_{j,i} over pairs without k."""
    dims = (3, 2, 4, 3)
    edge = {(0, 1): 2, (0, 2): 3, (0, 3): 2, (1, 2): 1, (1, 3): 2, (2, 3): 3}
    R, G = _problem(dims, edge, 40 + k)
    N = len(dims)
    F = inp.unpack_factors(G, dims, R)
    rest = [m for m in range(N) if m != k]
    S = np.ones([dims[m] for m in rest])
    for a_, i in enumerate(rest):
        for b_, j in enumerate(rest):
            if b_ <= a_:
                continue
            Wij = F[(i, j)].T @ F[(j, i)]
            shp = [1] * len(rest)
            shp[a_], shp[b_] = dims[i], dims[j]
            S = S * Wij.reshape(shp)
    K = None
    for i in range(N - 1, -1, -1):
        if i == k:
            continue
        K = F[(i, k)].T if K is None else np.kron(K, F[(i, k)].T)
    Z = S.reshape(-1, order="F")[:, None] * K
    core = _cherry_core(dims, R, F, k)
    Gk = _unfold_littleendian(core, k)  # I_k x prod R
    X = oracle.reconstruct(dims, R, G)
    np.testing.assert_allclose(Z @ Gk.T, _unfold_littleendian(X, k).T, rtol=1e-12, atol=1e-13)


def test_prop3_transposition_invariance():
    dims = (3, 4, 2, 5)
    edge = {(0, 1): 2, (0, 2): 3, (0, 3): 1, (1, 2): 2, (1, 3): 3, (2, 3): 2}
    R, G = _problem(dims, edge, 51)
    F = inp.unpack_factors(G, dims, R)
    X = oracle.reconstruct(dims, R, G)
    for n in [(2, 0, 3, 1), (3, 2, 1, 0), (1, 0, 2, 3)]:
        dn = tuple(dims[m] for m in n)
        Rn = np.zeros((4, 4), dtype=np.int32)
        for a in range(4):
            for b in range(4):
                if a != b:
                    Rn[a, b] = R[n[a], n[b]]
        Gn = np.concatenate([F[(n[k], n[l])].ravel() for k in range(4) for l in range(4) if l != k])
        np.testing.assert_allclose(oracle.reconstruct(dn, Rn, Gn), np.transpose(X, n),
                                   rtol=1e-13, atol=1e-14)


def test_reconstruction_invariant_under_edge_gauge():
    """Each rank index r_{k,l} appears only in G_{k,l} and G_{l,k} (eq. (iFCTN)), so
    G_{k,l} -> A G_{k,l}, G_{l,k} -> A^{-T} G_{l,k} with any invertible A leaves the
    tensor unchanged; the permutation-and-scaling ambiguity of Prop. 2 is the
    special case A = Pi Lambda.  A mispaired or transposed factor breaks it."""
    dims = (3, 4, 2, 3)
    edge = {(0, 1): 2, (0, 2): 3, (0, 3): 2, (1, 2): 3, (1, 3): 1, (2, 3): 2}
    R, G = _problem(dims, edge, 64)
    X = oracle.reconstruct(dims, R, G)
    rng = np.random.default_rng(65)
    G2 = G.copy()
    F2 = inp.unpack_factors(G2, dims, R)
    for (k, l), r in edge.items():
        A = rng.standard_normal((r, r)) + 2.0 * np.eye(r)
        F2[(k, l)][:, :] = A @ F2[(k, l)]
        F2[(l, k)][:, :] = np.linalg.inv(A).T @ F2[(l, k)]
    assert np.max(np.abs(G2 - G)) > 1e-2
    np.testing.assert_allclose(oracle.reconstruct(dims, R, G2), X, rtol=1e-11, atol=1e-12 * np.abs(X).max())
    # the same (not the inverse) scaling on both ends of an edge scales the tensor
    G3 = G.copy()
    F3 = inp.unpack_factors(G3, dims, R)
    F3[(0, 2)][:, :] = 2.0 * F3[(0, 2)]
    F3[(2, 0)][:, :] = 2.0 * F3[(2, 0)]
    assert np.max(np.abs(oracle.reconstruct(dims, R, G3) - X)) > 1e-3 * np.abs(X).max()


def test_rank_one_is_cp_outer_product():
    dims = (3, 4, 5, 2)
    R, G = _problem(dims, 1, 61)
    F = inp.unpack_factors(G, dims, R)
    u = [np.prod([F[(k, l)][0] for l in range(4) if l != k], axis=0) for k in range(4)]
    ref = np.einsum("i,j,k,l->ijkl", *u)
    np.testing.assert_allclose(oracle.reconstruct(dims, R, G), ref, rtol=1e-13, atol=1e-15)


def test_table5_parameter_count():
    (row,) = _golden("table5_parameter_count.txt")
    I1, I2, I3, r12, r13, r23, n_ifctn, n_fctn = map(int, row)
    R = inp.rank_matrix(3, {(0, 1): r12, (0, 2): r13, (1, 2): r23})
    assert oracle.param_count((I1, I2, I3), R) == n_ifctn
    assert inp.factor_size((I1, I2, I3), R) == n_ifctn
    # an FCTN core k holds I_k * prod_{l != k} R_{k,l} entries (eq. FCTN)
    fctn = sum(d * np.prod([R[k][l] for l in range(3) if l != k]) for k, d in enumerate((I1, I2, I3)))
    assert fctn == n_fctn


def test_table6_observed_rows_pin_metric_conventions():
    """RSE of the zero-filled observation = sqrt(missing fraction) and constant
    RMSE over missing entries: the printed Observed rows of Table 6."""
    rows = _golden("table6_observed_rows.txt")
    shape = (214, 61, 144)  # Guangzhou traffic tensor shape (Sec. 5.3)
    xt = 0.5 + 0.1 * inp.normal(77, int(np.prod(shape))).reshape(shape)
    rmses = []
    for _, miss, rse_printed, _rmse_printed in rows:
        miss = float(miss)
        mask = inp.uniform_mask(shape, 1.0 - miss, 78)
        Xobs = oracle.init_x(xt, mask)
        rse, rmse = oracle.metrics(xt, Xobs, mask)
        assert abs(rse - float(rse_printed)) < 1.5e-3, (miss, rse, rse_printed)
        rmses.append(rmse)
    assert max(rmses) - min(rmses) < 2e-3 * max(rmses)


# ---------------------------------------------------------------------------
# block update, eq. (updateG)
# ---------------------------------------------------------------------------

def _explicit_A(dims, R, G, k, i, j):
    """Dense coefficient matrix of column j of G_{k,i}: the model is linear in
    that column, so column r of A is the slice i_k = j of the reconstruction
    with the column set to e_r (computed by the FCTN route, not the oracle)."""
    F = inp.unpack_factors(G.copy(), dims, R)
    cols = []
    for r in range(int(R[k][i])):
        Gm = G.copy()
        Fm = inp.unpack_factors(Gm, dims, R)
        Fm[(k, i)][:, j] = 0.0
        Fm[(k, i)][r, j] = 1.0
        cores = [_cherry_core(dims, R, Fm, m) for m in range(len(dims))]
        Xr = _fctn_contract(dims, cores)
        cols.append(np.take(Xr, j, axis=k).ravel())
    del F
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("k,i,j", [(0, 1, 2), (1, 0, 0), (2, 1, 3), (3, 0, 1), (1, 3, 2)])
def test_block_system_equals_dense_normal_equations(k, i, j):
    dims = (3, 4, 5, 2)
    edge = {(0, 1): 2, (0, 2): 3, (0, 3): 2, (1, 2): 2, (1, 3): 3, (2, 3): 1}
    _check_block_system(dims, edge, k, i, j)


@pytest.mark.parametrize("k,i,j", [(0, 1, 2), (1, 0, 0), (2, 0, 3), (1, 2, 1)])
def test_block_system_equals_dense_normal_equations_ranks_above_eight(k, i, j):
    """The block buffers of the oracle hold ranks up to 64: the systems of
    edges of rank 12 and 36 (the largest R_{1,2} of the multispectral rank
    grid, Sec. 5.2) against the dense A_j of the FCTN route."""
    dims = (4, 3, 5)
    edge = {(0, 1): 36, (0, 2): 12, (1, 2): 9}
    _check_block_system(dims, edge, k, i, j)


def _check_block_system(dims, edge, k, i, j):
    R, G = _problem(dims, edge, 70 + k)
    X = inp.normal(71, int(np.prod(dims))).reshape(dims)
    A = _explicit_A(dims, R, G, k, i, j)
    x = np.take(X, j, axis=k).ravel()
    H, b = oracle.block_system(dims, R, G, X, k, i, j)
    np.testing.assert_allclose(H, A.T @ A, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b, A.T @ x, rtol=1e-12, atol=1e-12)


def _prop1_Z(dims, R, F, k):
    """Z_k of Prop. 1 (P_{-k} x Q_k): rows in the little-endian order of the
    remaining modes, columns the Kronecker order of kron_{m=N..1, m!=k} G_{m,k}^T."""
    N = len(dims)
    rest = [m for m in range(N) if m != k]
    S = np.ones([dims[m] for m in rest])
    for a_, p_ in enumerate(rest):
        for b_, q_ in enumerate(rest):
            if b_ <= a_:
                continue
            shp = [1] * len(rest)
            shp[a_], shp[b_] = dims[p_], dims[q_]
            S = S * (F[(p_, q_)].T @ F[(q_, p_)]).reshape(shp)
    K = None
    for m in range(N - 1, -1, -1):
        if m != k:
            K = F[(m, k)].T if K is None else np.kron(K, F[(m, k)].T)
    return S.reshape(-1, order="F")[:, None] * K


def _E(dims, R, F, k, i, j):
    """E_j: the Kronecker product, in Z_k's column order, of G_{k,m}(:, j) for
    m not in {k, i} and the identity at position i, so that Z_k E_j g is the
    slice i_k = j of the model as a function of column j of G_{k,i}."""
    N = len(dims)
    E = None
    for m in range(N - 1, -1, -1):
        if m == k:
            continue
        f = np.eye(int(R[k][i])) if m == i else F[(k, m)][:, j][:, None]
        E = f if E is None else np.kron(E, f)
    return E


@pytest.mark.parametrize("dims,edge", [
    ((3, 4, 5, 2), {(0, 1): 2, (0, 2): 3, (0, 3): 2, (1, 2): 2, (1, 3): 3, (2, 3): 1}),
    ((4, 3, 5), {(0, 1): 3, (0, 2): 2, (1, 2): 4}),
    ((4, 3, 5), {(0, 1): 12, (0, 2): 3, (1, 2): 10}),
])
def test_regrouped_mode_systems_equal_block_systems(dims, edge):
    """The regrouping the GPU path relies on (Prop. 1 applied to eq. (updateG)):
    with M_k = X_(k) Z_k and K_k = Z_k^T Z_k, every block system of mode k is
    H = E_j^T K_k E_j and b = E_j^T M_k(j,:)^T, for every i != k and every j."""
    R, G = _problem(dims, edge, 90 + len(dims))
    X = inp.normal(91, int(np.prod(dims))).reshape(dims)
    F = inp.unpack_factors(G, dims, R)
    N = len(dims)
    for k in range(N):
        Z = _prop1_Z(dims, R, F, k)
        M = _unfold_littleendian(X, k) @ Z
        K = Z.T @ Z
        for i in range(N):
            if i == k:
                continue
            for j in range(dims[k]):
                E = _E(dims, R, F, k, i, j)
                H, b = oracle.block_system(dims, R, G, X, k, i, j)
                np.testing.assert_allclose(E.T @ K @ E, H, rtol=1e-12, atol=1e-12)
                np.testing.assert_allclose(E.T @ M[j], b, rtol=1e-12, atol=1e-12)


def _numpy_sweep(dims, R, rho, G, X, mask):
    """Algorithm 1, one sweep, from explicit dense systems (tiny sizes only)."""
    N = len(dims)
    G = G.copy()
    X = X.copy()
    for k in range(N):
        for i in range(N):
            if i == k:
                continue
            F = inp.unpack_factors(G, dims, R)
            newcols = []
            for j in range(dims[k]):
                A = _explicit_A(dims, R, G, k, i, j)
                x = np.take(X, j, axis=k).ravel()
                n = A.shape[1]
                g = np.linalg.solve(A.T @ A + rho * np.eye(n), A.T @ x + rho * F[(k, i)][:, j])
                newcols.append(g)
            F[(k, i)][:, :] = np.stack(newcols, axis=1)
    cores = [_cherry_core(dims, R, inp.unpack_factors(G, dims, R), m) for m in range(N)]
    rec = _fctn_contract(dims, cores)
    Xn = np.where(mask.astype(bool), X, (rec + rho * X) / (1 + rho))
    return G, Xn


def test_sweep_equals_dense_gauss_seidel_pam():
    dims = (3, 2, 4)
    R, G0 = _problem(dims, {(0, 1): 2, (0, 2): 1, (1, 2): 2}, 81)
    xt = inp.normal(82, int(np.prod(dims))).reshape(dims)
    mask = inp.uniform_mask(dims, 0.6, 83)
    X0 = oracle.init_x(xt, mask)
    Gref, Xref = _numpy_sweep(dims, R, 0.3, G0, X0, mask)
    G = G0.copy()
    X = X0.copy()
    oracle.sweep(dims, R, 0.3, G, X, mask)
    np.testing.assert_allclose(G, Gref, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(X, Xref, rtol=1e-10, atol=1e-12)


def test_sweep_equals_dense_gauss_seidel_pam_ranks_above_eight():
    dims = (3, 2, 4)
    R, G0 = _problem(dims, {(0, 1): 10, (0, 2): 3, (1, 2): 12}, 84)
    xt = inp.normal(85, int(np.prod(dims))).reshape(dims)
    mask = inp.uniform_mask(dims, 0.6, 86)
    X0 = oracle.init_x(xt, mask)
    Gref, Xref = _numpy_sweep(dims, R, 0.3, G0, X0, mask)
    G = G0.copy()
    X = X0.copy()
    oracle.sweep(dims, R, 0.3, G, X, mask)
    np.testing.assert_allclose(G, Gref, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(X, Xref, rtol=1e-9, atol=1e-11)


def test_rank_above_oracle_limit_is_refused():
    dims = (3, 2, 4)
    R, G = _problem(dims, {(0, 1): 2, (0, 2): 2, (1, 2): 2}, 87)
    R = np.array(R)
    R[0, 1] = R[1, 0] = 65
    X = np.zeros(dims)
    with pytest.raises(RuntimeError):
        oracle.sweep(dims, R, 0.3, np.zeros(oracle.param_count(dims, R)), X, np.ones(dims, np.uint8))


@pytest.mark.parametrize("rank", [3, 12])
def test_two_way_case_is_proximal_als(rank):
    """N = 2: X = G_{1,2}^T G_{2,1}; each block is textbook proximal ALS."""
    dims = (6, 5)
    R, G = _problem(dims, rank, 91)
    F = inp.unpack_factors(G, dims, R)
    A0, B0 = F[(0, 1)].copy(), F[(1, 0)].copy()
    X = inp.normal(92, 30).reshape(dims)
    mask = np.ones(dims, dtype=np.uint8)
    rho = 0.2
    A1 = np.linalg.solve(B0 @ B0.T + rho * np.eye(rank), B0 @ X.T + rho * A0)
    B1 = np.linalg.solve(A1 @ A1.T + rho * np.eye(rank), A1 @ X + rho * B0)
    Gw = G.copy()
    Xw = X.copy()
    oracle.sweep(dims, R, rho, Gw, Xw, mask)
    Fw = inp.unpack_factors(Gw, dims, R)
    np.testing.assert_allclose(Fw[(0, 1)], A1, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(Fw[(1, 0)], B1, rtol=1e-12, atol=1e-13)
    np.testing.assert_array_equal(Xw, X)  # fully observed: X is never changed


@pytest.mark.parametrize("n", [8, 40])
def test_cholesky_solver(n):
    rng = inp.normal(93, n * n).reshape(n, n)
    H = rng @ rng.T + 0.5 * np.eye(n)
    b = inp.normal(94, n)
    np.testing.assert_allclose(oracle.cholesky_solve(H, b), np.linalg.solve(H, b), rtol=1e-10)


# ---------------------------------------------------------------------------
# whole sweeps: Lemma 2, stationarity, fixed point
# ---------------------------------------------------------------------------

def test_sufficient_decrease_lemma2_every_sweep():
    dims = (8, 7, 6)
    R, Gt = _problem(dims, {(0, 1): 2, (0, 2): 3, (1, 2): 2}, 101)
    xt = oracle.reconstruct(dims, R, Gt)
    mask = inp.uniform_mask(dims, 0.4, 102)
    rho = 0.1
    G = inp.uniform_factors(dims, R, 103)
    X = oracle.init_x(xt, mask)
    F = oracle.objective(dims, R, G, X)
    for _ in range(8):
        G0, X0 = G.copy(), X.copy()
        oracle.sweep(dims, R, rho, G, X, mask)
        F1 = oracle.objective(dims, R, G, X)
        step = np.sum((G - G0) ** 2) + np.sum((X - X0) ** 2)
        assert F - F1 >= 0.5 * rho * step - 1e-12 * max(F, 1.0), (F, F1, step)
        F = F1


def test_first_order_conditions_hold_after_block():
    """First-order condition of each block (appendix, proof of Lemma 3):
    A^T(A g - x) + rho (g - g_old) = 0 for the updated column."""
    dims = (4, 3, 5)
    R, G0 = _problem(dims, {(0, 1): 2, (0, 2): 3, (1, 2): 2}, 111)
    X = inp.normal(112, 60).reshape(dims)
    mask = np.zeros(dims, dtype=np.uint8)
    rho = 0.25
    G = G0.copy()
    oracle.sweep(dims, R, rho, G, X.copy(), mask)
    # block (0,1) is the first block, computed from the initial state
    F0 = inp.unpack_factors(G0, dims, R)
    Fn = inp.unpack_factors(G, dims, R)
    for j in range(dims[0]):
        Gs = G0.copy()
        A = _explicit_A(dims, R, Gs, 0, 1, j)
        x = np.take(X, j, axis=0).ravel()
        g, g0 = Fn[(0, 1)][:, j], F0[(0, 1)][:, j]
        grad = A.T @ (A @ g - x) + rho * (g - g0)
        scale = np.linalg.norm(A.T @ x) + rho * np.linalg.norm(g0)
        assert np.linalg.norm(grad) <= 1e-12 * scale


def test_planted_truth_is_fixed_point_under_full_observation():
    dims = (6, 5, 4, 3)
    R, Gt = _problem(dims, 2, 121)
    xt = oracle.reconstruct(dims, R, Gt)
    mask = np.ones(dims, dtype=np.uint8)
    G, X = Gt.copy(), xt.copy()
    st = oracle.sweep(dims, R, 0.1, G, X, mask)
    np.testing.assert_allclose(G, Gt, rtol=1e-11, atol=1e-12)
    np.testing.assert_array_equal(X, xt)
    assert st["objective"] <= 1e-20 * np.sum(xt ** 2)


def test_perturbed_planted_start_converges_monotonically():
    dims = (7, 6, 5)
    R, Gt = _problem(dims, 2, 131)
    xt = oracle.reconstruct(dims, R, Gt)
    mask = np.ones(dims, dtype=np.uint8)
    G = Gt + 1e-3 * inp.normal(132, Gt.size)
    X = xt.copy()
    log = oracle.complete(dims, R, 0.1, G, X, mask, max_sweeps=30)
    obj = [s["objective"] for s in log]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(obj, obj[1:]))
    assert obj[-1] < 1e-3 * obj[0]


def test_theorem1_limit_is_a_critical_point():
    """Theorem 1 (with Lemmas 2 and 3): the bounded PAM sequence has finite
    length and converges to a critical point of F(G, X) = 1/2 ||X - iFCTN(G)||^2
    over X with P_Omega(X) = P_Omega(O).  On a noisy problem whose observed
    entries the model cannot fit (F > 0 at the limit), run to a tight
    tolerance: the partial gradient of F in every factor column,
    A_j^T (A_j g - x_j), vanishes, X equals the reconstruction off Omega, and
    the steps ||X^{s+1} - X^s|| have a vanishing tail sum."""
    from tests._cases import make_case
    case = make_case((6, 5, 4), 2, 0.8, seed=111, kind="minmax01", sigma=0.05)
    dims, R, mask = case["dims"], case["R"], case["mask"]
    G, X = case["G0"].copy(), case["X0"].copy()
    log = oracle.complete(dims, R, 0.1, G, X, mask, max_sweeps=20000, tol=1e-12)
    assert len(log) < 20000 and log[-1]["rel_change"] < 1e-12
    assert log[-1]["objective"] > 1e-3                      # not an exact fit: a non-trivial critical point
    rec = oracle.reconstruct(dims, R, G)
    off = ~mask.astype(bool)
    assert np.linalg.norm((X - rec)[off]) < 1e-10 * np.linalg.norm(X)
    assert (X[~off] == case["X0"][~off]).all()
    F = inp.unpack_factors(G, dims, R)
    for k in range(3):
        for i in range(3):
            if i == k:
                continue
            for j in range(dims[k]):
                H, b = oracle.block_system(dims, R, G, X, k, i, j)
                g = F[(k, i)][:, j]
                assert np.linalg.norm(H @ g - b) <= 1e-9 * np.linalg.norm(b)
    steps = np.sqrt([s["dx2"] for s in log])
    assert steps[len(steps) // 2:].sum() < 1e-3 * steps.sum()


def test_observed_entries_unchanged_and_update_closed_form():
    dims = (5, 4, 6)
    R, G = _problem(dims, 2, 141)
    xt = inp.normal(142, 120).reshape(dims)
    mask = inp.uniform_mask(dims, 0.5, 143)
    X = oracle.init_x(xt, mask)
    X0 = X.copy()
    G1 = G.copy()
    oracle.sweep(dims, R, 0.1, G1, X, mask)
    rec = oracle.reconstruct(dims, R, G1)
    obs = mask.astype(bool)
    np.testing.assert_array_equal(X[obs], X0[obs])
    np.testing.assert_allclose(X[~obs], (rec[~obs] + 0.1 * X0[~obs]) / 1.1, rtol=1e-14, atol=1e-15)
    np.testing.assert_array_equal(X0[~obs], 0.0)  # X^0 = P_Omega(O)


def test_thread_count_does_not_change_results():
    dims = (9, 8, 7)
    R, G = _problem(dims, 3, 151)
    xt = inp.normal(152, int(np.prod(dims))).reshape(dims)
    mask = inp.uniform_mask(dims, 0.3, 153)
    outs = []
    for nt in (1, 4):
        Gw, Xw = G.copy(), oracle.init_x(xt, mask)
        oracle.sweep(dims, R, 0.1, Gw, Xw, mask, nthreads=nt)
        outs.append((Gw, Xw))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


# ---------------------------------------------------------------------------
# the objective of Sec. 4.1, eq. (iFCTN-TC): F = 1/2 ||X - iFCTN(G)||_F^2
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,edge,seed", [
    ((5, 4, 6), {(0, 1): 2, (0, 2): 3, (1, 2): 2}, 131),
    ((3, 4, 2, 3), {(0, 1): 2, (0, 2): 1, (0, 3): 2, (1, 2): 3, (1, 3): 2, (2, 3): 1}, 132),
])
def test_objective_is_half_squared_misfit_of_the_fctn_contraction(dims, edge, seed):
    """The objective of eq. (iFCTN-TC) written out independently of the oracle:
    the reconstruction is the eq. (FCTN) contraction of the Def. 1 cherry
    cores, the misfit is taken against the tensor after the X block of the
    sweep (X^{s+1}) and the factors after it (G^{s+1}), and the weight is 1/2.
    A dropped 1/2, a misfit against X^s or against the factors before the
    sweep each moves the value by far more than the tolerance."""
    N = len(dims)
    R, Gt = _problem(dims, edge, seed)
    xt = oracle.reconstruct(dims, R, Gt) + 0.05 * inp.normal(seed + 1, int(np.prod(dims))).reshape(dims)
    mask = inp.uniform_mask(dims, 0.5, seed + 2)
    G = inp.uniform_factors(dims, R, seed + 3)
    X = oracle.init_x(xt, mask)

    def f_ref(Gv, Xv):
        F = inp.unpack_factors(Gv, dims, R)
        rec = _fctn_contract(dims, [_cherry_core(dims, R, F, m) for m in range(N)])
        return 0.5 * float(np.sum((Xv - rec) ** 2))

    assert oracle.objective(dims, R, G, X) == pytest.approx(f_ref(G, X), rel=1e-12)
    for _ in range(2):
        Gs, Xs = G.copy(), X.copy()
        st = oracle.sweep(dims, R, 0.1, G, X, mask)
        want = f_ref(G, X)
        assert st["objective"] == pytest.approx(want, rel=1e-12)
        assert oracle.objective(dims, R, G, X) == pytest.approx(want, rel=1e-12)
        # the pin separates the readings it rules out
        assert abs(f_ref(G, Xs) - want) > 1e-6 * want
        assert abs(f_ref(Gs, X) - want) > 1e-6 * want
