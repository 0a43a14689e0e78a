"""The biclique oracle (Sec. 6) against what fixes it independently: a
hand-worked example (tests/golden/biclique_example_n6.txt) and dense
brute force on random decompositions. No GPU needed."""
import os

import numpy as np

from oracle import biclique as ob

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "biclique_example_n6.txt")


def read_golden():
    s, c, res, vals = [], [], [], {}
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        key, *rest = line.split()
        if key == "s":
            s.append([int(t) for t in rest])
        elif key == "c":
            c.append([int(t) for t in rest])
        elif key == "residual":
            res.append((int(rest[0]), int(rest[1])))
        else:
            vals[key] = [float(t) for t in rest]
    n = int(vals["n"][0])
    return n, s, c, res, vals


def make_dec(n, s_lists, c_lists, residual):
    s_ptr = np.zeros(len(s_lists) + 1, np.int64)
    s_ptr[1:] = np.cumsum([len(v) for v in s_lists])
    c_ptr = np.zeros(len(c_lists) + 1, np.int64)
    c_ptr[1:] = np.cumsum([len(v) for v in c_lists])
    rows = [sorted(j for i2, j in residual if i2 == i) for i in range(n)]
    r_ptr = np.zeros(n + 1, np.int64)
    r_ptr[1:] = np.cumsum([len(v) for v in rows])
    cat = lambda ls: np.array([t for v in ls for t in v], np.int32)  # noqa: E731
    return {"s_ptr": s_ptr, "s_idx": cat(s_lists), "c_ptr": c_ptr, "c_idx": cat(c_lists),
            "r_ptr": r_ptr, "r_col": cat(rows)}


def dense_of(dec, n):
    a = np.zeros((n, n))
    for e in ob.edges_of(dec, n):
        a[e // n, e % n] += 1.0
    return a


def test_hand_worked_example():
    n, s, c, res, vals = read_golden()
    dec = make_dec(n, s, c, res)
    x = np.array(vals["x"])
    np.testing.assert_array_equal(ob.biclique_Ax(dec, x), vals["Ax"])
    np.testing.assert_array_equal(ob.biclique_xA(dec, x), vals["xA"])
    assert ob.words(dec) == int(vals["words"][0])
    assert len(ob.edges_of(dec, n)) == int(vals["m"][0])


def test_random_decompositions_match_dense_brute_force():
    rng = np.random.default_rng(1708)
    for trial in range(20):
        n = int(rng.integers(2, 40))
        nb = int(rng.integers(0, 5))
        used = set()
        s_lists, c_lists = [], []
        for _ in range(nb):
            s = sorted(rng.choice(n, size=int(rng.integers(1, n + 1)), replace=False).tolist())
            c = sorted(rng.choice(n, size=int(rng.integers(1, n + 1)), replace=False).tolist())
            c = [j for j in c if all((i, j) not in used for i in s)]  # bicliques stay edge-disjoint
            if not c:
                continue
            used.update((i, j) for i in s for j in c)
            s_lists.append(s)
            c_lists.append(c)
        residual = [(i, j) for i in range(n) for j in range(n) if (i, j) not in used and rng.random() < 0.15]
        dec = make_dec(n, s_lists, c_lists, residual)
        a = dense_of(dec, n)
        assert a.max() <= 1.0  # edge-disjoint: a binary matrix
        x = rng.integers(-8, 9, size=(n, 3)).astype(np.float64) / 8.0  # dyadic: exact sums
        np.testing.assert_array_equal(ob.biclique_Ax(dec, x), a @ x)
        np.testing.assert_array_equal(ob.biclique_xA(dec, x), a.T @ x)  # (x A)^T = A^T x^T
