"""ORACLE -- test infrastructure only.

Plain FP64 reference of the warm-start network 6 -> 64 -> 64 -> 1 (ReLU) and
of its node features, for checking the GPU kernels. Not from the paper: the
paper's method has no learned part; this network predicts a starting vector
for the PageRank power iteration (Eq. 1), whose fixed point does not depend
on the start.

Parameter vector layout (4673 FP32 values):
  W1 [64][6], b1 [64], W2 [64][64], b2 [64], w3 [64], b3 [1]
Forward, as computed on the GPU (quantize=True):
  a1 = bf16(W1) f + b1;  h1 = relu(a1);  h1q = bf16(h1)
  a2 = bf16(W2) h1q + b2; h2 = relu(a2);  yhat = bf16(w3) . h2 + b3
Loss (mean squared error over N nodes): L = sum_i (yhat_i - t_i)^2 / N,
with the target t_i = n p*_i (the PageRank vector scaled to mean 1).
Backward: the rounding steps pass gradients through unchanged.
With quantize=False every step is exact FP64 (used for the finite-difference
pin of the backward formulas).
"""
from __future__ import annotations

import numpy as np

H = 64
NF = 6
SIZES = [("W1", (H, NF)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + k], np.float64).reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SIZES])


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), through FP32."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def forward(theta, f, quantize=True):
    p = unpack(theta)
    q = bf16 if quantize else (lambda a: np.asarray(a, np.float64))
    f = np.asarray(f, np.float64)[:, :NF]
    a1 = f @ q(p["W1"]).T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    h1q = q(h1)
    a2 = h1q @ q(p["W2"]).T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    yhat = h2 @ q(p["w3"]) + p["b3"][0]
    return yhat, (f, a1, h1q, a2, h2, p, q)


def loss_grad(theta, f, t, quantize=True):
    """Mean squared error and its gradient with respect to theta."""
    yhat, (f, a1, h1q, a2, h2, p, q) = forward(theta, f, quantize)
    n = len(yhat)
    r = yhat - np.asarray(t, np.float64)
    loss = float(np.sum(r * r) / n)
    dy = 2.0 * r / n
    g = {}
    g["w3"] = h2.T @ dy
    g["b3"] = np.array([dy.sum()])
    dh2 = np.outer(dy, q(p["w3"])) * (a2 > 0)
    g["W2"] = dh2.T @ h1q
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ q(p["W2"])) * (a1 > 0)
    g["W1"] = dh1.T @ f
    g["b1"] = dh1.sum(axis=0)
    return loss, pack(g)


def init(seed):
    """He-style initial weights (a host-side choice shared with the GPU tests)."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, np.sqrt(2.0 / NF), (H, NF)), "b1": np.zeros(H),
         "W2": rng.normal(0, np.sqrt(2.0 / H), (H, H)), "b2": np.zeros(H),
         "w3": rng.normal(0, np.sqrt(1.0 / H), H), "b3": np.zeros(1)}
    return pack(d).astype(np.float32)


def features(row_ptr, col, ref, depth, min_interval=4):
    """Node features, FP64, by definition:
    log1p(in-degree), log1p(out-degree), reference-chain depth, fraction of the
    row's successors that its difference row stores as intervals, log1p(mean
    out-degree of the successors), log1p(weighted in-degree), where the
    weighted in-degree of i is sum over edges j -> i of 1/outdeg(j) (the
    share of uniform mass one step of Eq. 1 without teleport brings to i)."""
    rp = np.asarray(row_ptr, np.int64)
    ci = np.asarray(col, np.int64)
    n = len(rp) - 1
    outdeg = np.diff(rp).astype(np.float64)
    indeg = np.bincount(ci, minlength=n).astype(np.float64)
    nbr = np.zeros(n)
    np.add.at(nbr, np.repeat(np.arange(n), np.diff(rp)), outdeg[ci])
    mean_nbr = np.where(outdeg > 0, nbr / np.maximum(outdeg, 1), 0.0)
    ivfrac = np.zeros(n)
    for i in range(n):
        vi = ci[rp[i]:rp[i + 1]]
        r = ref[i]
        vr = set(ci[rp[r]:rp[r + 1]].tolist()) if r >= 0 else set()
        added = [j for j in vi.tolist() if j not in vr]
        members, run = 0, []
        for j in added + [None]:
            if run and (j is None or j != run[-1] + 1):
                if len(run) >= min_interval:
                    members += len(run)
                run = []
            if j is not None:
                run.append(j)
        ivfrac[i] = members / outdeg[i] if outdeg[i] > 0 else 0.0
    f = np.zeros((n, 8))
    f[:, 0] = np.log1p(indeg)
    f[:, 1] = np.log1p(outdeg)
    f[:, 2] = np.asarray(depth, np.float64)
    f[:, 3] = ivfrac
    f[:, 4] = np.log1p(mean_nbr)
    src = np.repeat(np.arange(n), np.diff(rp))
    wdeg = np.bincount(ci, weights=1.0 / outdeg[src], minlength=n) if len(ci) else np.zeros(n)
    f[:, 5] = np.log1p(wdeg)
    return f
