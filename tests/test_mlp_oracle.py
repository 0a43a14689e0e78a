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


def _golden_theta(g):
    """The parameter vector of the hand-worked example (zeros elsewhere)."""
    p = {name: np.zeros(shape) for name, shape in mlp.SIZES}
    for u in range(3):
        p["W1"][u] = [float(v) for v in g[f"W1_{u}"]]
    p["b1"][:3] = [float(v) for v in g["b1_012"]]
    for u in range(2):
        p["W2"][u, :3] = [float(v) for v in g[f"W2_{u}_012"]]
    p["b2"][:2] = [float(v) for v in g["b2_01"]]
    p["w3"][:2] = [float(v) for v in g["w3_01"]]
    p["b3"][0] = float(g["b3"][0])
    return mlp.pack(p)


def test_forward_on_hand_worked_example():
    """The forward map against values worked out by hand: the bias of every
    layer, ReLU before the bfloat16 rounding of the first hidden layer (a tie
    rounded to even), the rounding of a weight (a tie), and the output bias
    added after the output product; and the same network without rounding."""
    g = load_golden("mlp_forward_n2.txt")
    theta = _golden_theta(g)
    f = np.array([[float(v) for v in g["f_A"]] + [0, 0], [float(v) for v in g["f_B"]] + [0, 0]])
    yq, _ = mlp.forward(theta, f, quantize=True)
    np.testing.assert_array_equal(yq, [float(v) for v in g["yhat_bf16"]])
    y64, _ = mlp.forward(theta, f, quantize=False)
    np.testing.assert_array_equal(y64, [float(v) for v in g["yhat_fp64"]])


def test_forward_matches_torch_layers():
    """The forward map against a network assembled from torch.nn layers in
    FP64 (nn.Linear, nn.ReLU) from the same parameter layout, with torch's own
    bfloat16 conversion for the rounding steps: random weights and inputs."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    theta = mlp.init(11).astype(np.float64)
    theta += rng.normal(0, 0.05, theta.shape)  # nonzero biases too
    f = rng.normal(0, 1.5, (300, 8))
    p = mlp.unpack(theta)

    def rnd(a):
        return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64)

    for quantize in (True, False):
        q = rnd if quantize else (lambda a: torch.as_tensor(a, dtype=torch.float64))
        l1 = torch.nn.Linear(mlp.NF, mlp.H).double()
        l2 = torch.nn.Linear(mlp.H, mlp.H).double()
        l3 = torch.nn.Linear(mlp.H, 1).double()
        with torch.no_grad():
            l1.weight.copy_(q(p["W1"]))
            l1.bias.copy_(torch.as_tensor(p["b1"]))
            l2.weight.copy_(q(p["W2"]))
            l2.bias.copy_(torch.as_tensor(p["b2"]))
            l3.weight.copy_(q(p["w3"]).reshape(1, -1))
            l3.bias.copy_(torch.as_tensor(p["b3"]))
            h1 = torch.nn.ReLU()(l1(torch.as_tensor(f[:, :mlp.NF])))
            h1 = rnd(h1.numpy().astype(np.float32)) if quantize else h1
            want = l3(torch.nn.ReLU()(l2(h1))).reshape(-1).numpy()
        got, _ = mlp.forward(theta, f, quantize=quantize)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
