"""Pins of the warm-start network oracle (oracle/mlp.py): the backward
formulas against central finite differences, the bfloat16 rounding against
PyTorch's conversion, and the node features on the hand-worked example."""
import numpy as np
import pytest

from oracle import mlp
from conftest import load_golden


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init(3).astype(np.float64)
    theta[mlp.NPARAM - 1] = 0.3
    f = rng.normal(0, 1, (40, 8))
    t = rng.normal(0, 1, 40)
    loss, g = mlp.loss_grad(theta, f, t, quantize=False)
    h = 1e-6
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    fd = np.empty(len(idx))
    for j, p in enumerate(idx):
        e = np.zeros(mlp.NPARAM)
        e[p] = h
        fd[j] = (mlp.loss_grad(theta + e, f, t, False)[0] - mlp.loss_grad(theta - e, f, t, False)[0]) / (2 * h)
    assert np.linalg.norm(fd - g[idx]) <= 1e-6 * max(1.0, np.linalg.norm(fd))
    # the bias gradient of the output is exactly 2 mean(residual)
    yhat, _ = mlp.forward(theta, f, quantize=False)
    assert g[-1] == pytest.approx(2 * np.mean(yhat - t), rel=1e-12)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -2.5, 1e-3, 3.14159, 65504.0, 2 ** -130, 0.0],
                    np.float32)
    want = torch.tensor(vals).to(torch.bfloat16).float().numpy().astype(np.float64)
    np.testing.assert_array_equal(mlp.bf16(vals), want)
    assert mlp.bf16(np.float32(1 + 2 ** -8)) == 1.0  # tie to even


def test_features_on_worked_example():
    g = load_golden("worked_example_n8.txt")
    lists = [[2, 3, 4, 5], [2, 3, 4, 5, 7], [0, 3, 4, 5, 7], [], [0, 3, 4, 5, 6, 7], [0, 3, 4, 5, 6, 7], [1],
             [1, 6]]
    rp = np.zeros(9, np.int64)
    rp[1:] = np.cumsum([len(v) for v in lists])
    col = np.array([j for v in lists for j in v], np.int32)
    ref = np.array([int(v) for v in g["ref"]])
    depth = np.array([int(v) for v in g["depth"]])
    f = mlp.features(rp, col, ref, depth)
    # in/out-degrees and successor mean out-degrees worked out by hand
    indeg = [3, 2, 2, 5, 5, 5, 3, 4]
    outdeg = [4, 5, 5, 0, 6, 6, 1, 2]
    mean_nbr = [17 / 4, 19 / 5, 18 / 5, 0, 19 / 6, 19 / 6, 5, 3]
    np.testing.assert_allclose(f[:, 0], np.log1p(indeg))
    np.testing.assert_allclose(f[:, 1], np.log1p(outdeg))
    np.testing.assert_array_equal(f[:, 2], depth)
    np.testing.assert_array_equal(f[:, 3], [1, 0, 0, 0, 0, 0, 0, 0])  # only row 0 stores an interval
    np.testing.assert_allclose(f[:, 4], np.log1p(mean_nbr))
    # weighted in-degree sum_{j -> i} 1/outdeg(j), by hand; it sums to the 7 non-dangling rows
    wdeg = [8 / 15, 3 / 2, 9 / 20, 59 / 60, 59 / 60, 59 / 60, 5 / 6, 11 / 15]
    assert abs(sum(wdeg) - 7) < 1e-12
    np.testing.assert_allclose(f[:, 5], np.log1p(wdeg))
