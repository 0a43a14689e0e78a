"""Pins of the CPU oracle to things other than itself (no GPU needed).

- a hand-worked example (tests/golden/worked_example_n8.txt);
- dense brute force with NumPy on tiny graphs, exact with dyadic inputs;
- Proposition 1: the compressed product equals the plain one for ANY valid
  reference vector, not only the chosen one;
- sum identities sum(xA) = sum_i x_i outdeg(i), sum(Ax) = sum_j x_j indeg(j);
- the reference-choice rule re-derived with Python sets on tiny graphs;
- PageRank: total mass 1, the dense linear solve, closed forms, linearity in
  the teleport vector, the (1 - alpha) contraction and start independence.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.dense import dense_matrix, pagerank_solve
from conftest import load_golden


def random_graph(n, density, seed, local=False):
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        if local:
            cand = np.arange(max(0, i - 6), min(n, i + 7))
            pick = cand[rng.random(len(cand)) < density]
        else:
            pick = np.nonzero(rng.random(n) < density)[0]
        rows.append(np.unique(pick))
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32) if rp[-1] else np.zeros(0, np.int32)
    return rp, col


def copy_graph(n, seed):
    """Tiny copying-model graph: exercises references, drops and intervals."""
    g = synth.copying_model(synth.GraphSpec(n=n, seed=seed, p_copy=0.7, fidelity=0.8, extra_mean=1.0,
                                            fresh_mean=6.0, q_run=0.4, gap_mean=4.0))
    return g.row_ptr, g.col


def dyadic(n, k, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 64, size=(n, k)).astype(np.float64) / 1024.0


# --------------------------------------------------------------- golden
def test_worked_example():
    g = load_golden("worked_example_n8.txt")
    lists = [[2, 3, 4, 5], [2, 3, 4, 5, 7], [0, 3, 4, 5, 7], [], [0, 3, 4, 5, 6, 7], [0, 3, 4, 5, 6, 7], [1],
             [1, 6]]
    rp = np.zeros(9, np.int64)
    rp[1:] = np.cumsum([len(v) for v in lists])
    col = np.array([j for v in lists for j in v], np.int32)
    ref, depth = oracle.choose_refs(rp, col, window=7, max_chain=3, min_interval=4)
    assert ref.tolist() == [int(v) for v in g["ref"]]
    assert depth.tolist() == [int(v) for v in g["depth"]]
    want = dict(kv.split("=") for kv in g["counts"])
    got = oracle.counts(rp, col, ref, 4)
    assert {k: str(v) for k, v in got.items()} == want
    x = np.array([float(v) for v in g["x"]])
    assert oracle.csr_Ax(rp, col, x).tolist() == [float(v) for v in g["Ax"]]
    assert oracle.bv_Ax(rp, col, ref, x).tolist() == [float(v) for v in g["Ax"]]
    assert oracle.csr_xA(rp, col, x).tolist() == [float(v) for v in g["xA"]]
    assert oracle.bv_xA(rp, col, ref, x).tolist() == [float(v) for v in g["xA"]]
    assert oracle.chain_weights(ref, x).tolist() == [float(v) for v in g["z"]]


# --------------------------------------------------------------- dense brute force
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("kind", ["random", "local", "copy"])
def test_products_equal_dense(seed, kind):
    n = 48
    if kind == "copy":
        rp, col = copy_graph(n, 1000 + seed)
    else:
        rp, col = random_graph(n, 0.15 if kind == "random" else 0.5, seed, local=(kind == "local"))
    A = dense_matrix(rp, col)
    assert not np.array_equal(A, A.T) or A.sum() == 0
    x = dyadic(n, 3, seed)
    np.testing.assert_array_equal(oracle.csr_Ax(rp, col, x), A @ x)
    np.testing.assert_array_equal(oracle.csr_xA(rp, col, x), A.T @ x)
    ref, _ = oracle.choose_refs(rp, col)
    np.testing.assert_array_equal(oracle.bv_Ax(rp, col, ref, x), A @ x)
    np.testing.assert_array_equal(oracle.bv_xA(rp, col, ref, x), A.T @ x)


@pytest.mark.parametrize("seed", range(8))
def test_proposition1_any_reference(seed):
    """A x = A' x + w holds for every reference vector with r_i < i (the
    window and chain bound are encoder choices, not conditions of the
    identity), so arbitrary references must give the plain product."""
    n = 40
    rp, col = random_graph(n, 0.4, 50 + seed, local=True)
    rng = np.random.default_rng(seed)
    ref = np.array([-1 if i == 0 or rng.random() < 0.2 else int(rng.integers(0, i)) for i in range(n)], np.int32)
    A = dense_matrix(rp, col)
    x = dyadic(n, 2, seed + 7)
    np.testing.assert_array_equal(oracle.bv_Ax(rp, col, ref, x), A @ x)
    np.testing.assert_array_equal(oracle.bv_xA(rp, col, ref, x), A.T @ x)
    # z_k: sum of x over the rows whose chain passes through k (brute force)
    z = np.zeros_like(x)
    for i in range(n):
        k = i
        while k >= 0:
            z[k] += x[i]
            k = ref[k]
    np.testing.assert_array_equal(oracle.chain_weights(ref, x), z)


def test_sum_identities():
    g = synth.copying_model(synth.tiny_web())
    x = synth.rhs(g.n, 2, synth.seed_for(1, 1)).astype(np.float64)
    outdeg = np.diff(g.row_ptr)
    indeg = np.bincount(g.col, minlength=g.n)
    ref, _ = oracle.choose_refs(g.row_ptr, g.col)
    for y in (oracle.csr_xA(g.row_ptr, g.col, x), oracle.bv_xA(g.row_ptr, g.col, ref, x)):
        np.testing.assert_allclose(y.sum(axis=0), (x * outdeg[:, None]).sum(axis=0), rtol=1e-12)
    for y in (oracle.csr_Ax(g.row_ptr, g.col, x), oracle.bv_Ax(g.row_ptr, g.col, ref, x)):
        np.testing.assert_allclose(y.sum(axis=0), (x * indeg[:, None]).sum(axis=0), rtol=1e-12)


# --------------------------------------------------------------- reference choice
def _cost_sets(vi, vr, lmin):
    dropped = len(vr - vi)
    added = sorted(vi - vr)
    res = ints = 0
    run = []
    for j in added + [None]:
        if run and (j is None or j != run[-1] + 1):
            if len(run) >= lmin:
                ints += 1
            else:
                res += len(run)
            run = []
        if j is not None:
            run.append(j)
    return dropped + res + 2 * ints, len(vr ^ vi), dropped, res, ints


def _choose_sets(lists, W, R, lmin):
    n = len(lists)
    ref, depth = [-1] * n, [0] * n
    for i in range(n):
        vi = set(lists[i])
        raw = _cost_sets(vi, set(), lmin)[0]
        best = None
        for r in range(i - 1, max(-1, i - W - 1), -1):
            if depth[r] >= R:
                continue
            cost, sym, *_ = _cost_sets(vi, set(lists[r]), lmin)
            if best is None or cost < best[0]:
                best = (cost, r, sym)
        if best is not None and best[0] < raw and best[2] < len(vi):
            ref[i], depth[i] = best[1], depth[best[1]] + 1
    return ref, depth


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("W,R,lmin", [(7, 3, 4), (3, 1, 2), (7, 2, 3)])
def test_choose_refs_matches_set_brute_force(seed, W, R, lmin):
    n = 60
    rp, col = copy_graph(n, 77 + seed)
    lists = [col[rp[i]:rp[i + 1]].tolist() for i in range(n)]
    ref, depth = oracle.choose_refs(rp, col, W, R, lmin)
    want_ref, want_depth = _choose_sets(lists, W, R, lmin)
    assert ref.tolist() == want_ref
    assert depth.tolist() == want_depth
    # invariants: window, chain bound, keep-raw rule of Sec. 5
    for i in range(n):
        if ref[i] >= 0:
            assert i - W <= ref[i] < i
            assert len(set(lists[i]) ^ set(lists[ref[i]])) < len(lists[i])
        assert depth[i] <= R
    # counts re-derived with sets
    tot = np.zeros(3, np.int64)
    for i in range(n):
        vr = set(lists[ref[i]]) if ref[i] >= 0 else set()
        _, _, d, r_, k_ = _cost_sets(set(lists[i]), vr, lmin)
        tot += (d, r_, k_)
    c = oracle.counts(rp, col, ref, lmin)
    assert (c["dropped"], c["residual"], c["intervals"]) == tuple(int(v) for v in tot)


# --------------------------------------------------------------- PageRank
ALPHA = 0.15


def test_pagerank_two_node_closed_form():
    """0 -> 1, node 1 dangling, p0 uniform. The fixed point solves
    p0' = a/2 + (1-a) p1/2,  p1' = a/2 + (1-a)(p0' + p1/2),  p0' + p1' = 1,
    i.e. p0' = 1/(3-a), p1' = (2-a)/(3-a)."""
    rp = np.array([0, 1, 1], np.int64)
    col = np.array([1], np.int32)
    p, it, res = oracle.pagerank(rp, col, alpha=ALPHA, tol=1e-15, max_iter=10_000)
    np.testing.assert_allclose(p[:, 0], [1 / (3 - ALPHA), (2 - ALPHA) / (3 - ALPHA)], rtol=0, atol=1e-14)


def test_pagerank_cycle_and_empty():
    n = 37
    rp = np.arange(n + 1, dtype=np.int64)
    col = ((np.arange(n) + 1) % n).astype(np.int32)
    p, it, _ = oracle.pagerank(rp, col, alpha=ALPHA, tol=1e-15, max_iter=100)
    np.testing.assert_allclose(p[:, 0], 1.0 / n, rtol=1e-14)
    # empty graph: all mass is dangling and returns to p0 in one update
    rp0 = np.zeros(n + 1, np.int64)
    p0 = np.random.default_rng(0).random(n)
    p0 /= p0.sum()
    p, it, res = oracle.pagerank(rp0, np.zeros(0, np.int32), alpha=ALPHA, p0=p0, p_init=np.full(n, 1.0 / n),
                                 tol=1e-15, max_iter=5)
    np.testing.assert_allclose(p[:, 0], p0, rtol=1e-14)
    assert it == 2 and res[0] < 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_pagerank_dense_solve(seed):
    n = 150
    rp, col = random_graph(n, 0.012, 900 + seed)
    assert (np.diff(rp) == 0).any()  # has dangling nodes
    A = dense_matrix(rp, col)
    rng = np.random.default_rng(seed)
    p0 = rng.random(n)
    p0 /= p0.sum()
    for dangling in (0, 1):
        want = pagerank_solve(A, ALPHA, p0, dangling)
        p, it, res = oracle.pagerank(rp, col, alpha=ALPHA, p0=p0, tol=1e-14, max_iter=10_000, dangling=dangling)
        assert res[0] < 1e-14
        np.testing.assert_allclose(p[:, 0], want, rtol=0, atol=1e-12)
        assert abs(p.sum() - 1.0) < 1e-12


def test_pagerank_one_hot_columns_dense_solve():
    """Personalised PageRank with one-hot teleport vectors (e_s, the input
    form of bvg_pagerank_seeds), several columns in one run: each column is
    the dense linear solve for its own seed, for both dangling policies."""
    n = 150
    rp, col = random_graph(n, 0.012, 905)
    assert (np.diff(rp) == 0).any()
    A = dense_matrix(rp, col)
    seeds = np.array([0, 17, 17, 149, int(np.nonzero(np.diff(rp) == 0)[0][0])])  # a repeat, the last row, a dangling row
    P0 = np.zeros((n, len(seeds)))
    P0[seeds, np.arange(len(seeds))] = 1.0
    for dangling in (0, 1):
        p, it, res = oracle.pagerank(rp, col, alpha=ALPHA, p0=P0, tol=1e-14, max_iter=10_000, dangling=dangling)
        assert (res < 1e-14).all()
        for c, s in enumerate(seeds):
            e = np.zeros(n)
            e[s] = 1.0
            np.testing.assert_allclose(p[:, c], pagerank_solve(A, ALPHA, e, dangling), rtol=0, atol=1e-12)
        np.testing.assert_array_equal(p[:, 1], p[:, 2])


def test_pagerank_mass_linearity_contraction_start():
    g = synth.copying_model(synth.tiny_web())
    n = g.n
    p, it, res = oracle.pagerank(g.row_ptr, g.col, alpha=ALPHA, tol=1e-8, max_iter=20)
    assert it == 20
    assert abs(p.sum() - 1.0) < 1e-12  # no renormalisation inside
    pstar, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=ALPHA, tol=1e-14, max_iter=1000)
    # contraction: ||p_t - p*||_1 <= (1-alpha)^t ||p_0 - p*||_1
    p0 = np.full((n, 1), 1.0 / n)
    for t in (1, 5, 12):
        pt, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=ALPHA, tol=0.0, max_iter=t)
        assert np.abs(pt - pstar).sum() <= (1 - ALPHA) ** t * np.abs(p0 - pstar).sum() * (1 + 1e-9) + 1e-13
    # start independence
    rng = np.random.default_rng(3)
    start = rng.random(n)
    start /= start.sum()
    pw, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=ALPHA, p_init=start, tol=1e-14, max_iter=1000)
    assert np.abs(pw - pstar).sum() < 1e-12
    # personalized: with the dangling mass spread uniformly, the fixed point is
    # linear in the teleport vector; returning it along p0 makes the operator
    # itself depend on p0, and linearity must then fail (the graph has
    # dangling rows)
    assert (np.diff(g.row_ptr) == 0).any()
    seeds = synth.nodes(3, n, 11)
    P0 = np.zeros((n, 3))
    P0[seeds, np.arange(3)] = 1.0
    w = np.array([0.5, 0.3, 0.2])
    cols, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=ALPHA, p0=P0, tol=1e-14, max_iter=1000, dangling=1)
    mix, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=ALPHA, p0=P0 @ w, tol=1e-14, max_iter=1000, dangling=1)
    np.testing.assert_allclose(mix[:, 0], cols @ w, rtol=0, atol=1e-12)
    cols0, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=ALPHA, p0=P0, tol=1e-14, max_iter=1000)
    mix0, _, _ = oracle.pagerank(g.row_ptr, g.col, alpha=ALPHA, p0=P0 @ w, tol=1e-14, max_iter=1000)
    assert np.abs(mix0[:, 0] - cols0 @ w).max() > 1e-9
