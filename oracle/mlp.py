"""FP64 oracle of the pair-screening network (test infrastructure).

The conclusions of the paper (Sec. 5) propose screening electron pairs and
keeping only those that contribute meaningfully, which would cut the number of
pairs from N^2 towards N.  The paper gives no algorithm.  The learned screen
here predicts, for every localized-orbital pair [ij], the decimal log of the
largest exchange contribution |e_ij| over a set of training walkers from eight
walker-independent pair descriptors, and drops pairs predicted below a cutoff.

Network: x (8) -> tanh(W1 x + b1) (64) -> tanh(W2 h1 + b2) (64) -> W3 h2 + b3.
Loss: mean squared error over the training pairs.  Optimiser: Adam (Kingma and
Ba), full batch, lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8.  Inputs and
targets are standardised with the training set's mean and standard deviation
(a zero deviation counts as one).

Only the test suite, the smoke check and the CPU baseline of the benchmark use
this module.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List

import numpy as np

SHAPES = [("W1", (64, 8)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)),
          ("W3", (1, 64)), ("b3", (1,))]


def n_params() -> int:
    return sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> Dict[str, np.ndarray]:
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(p: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def standardise(x: np.ndarray):
    """Column mean and deviation (deviation 0 -> 1)."""
    mu = x.mean(axis=0)
    sd = x.std(axis=0)
    sd = np.where(sd > 0, sd, 1.0)
    return mu, sd


def forward(theta: np.ndarray, x: np.ndarray):
    """Predictions (n,) and the activations the backward pass needs."""
    p = unpack(theta)
    a1 = x @ p["W1"].T + p["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(a2)
    y = (h2 @ p["W3"].T + p["b3"])[:, 0]
    return y, (x, h1, h2)


def loss(theta: np.ndarray, x: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(theta, x)
    return float(np.mean((y - t) ** 2))


def grad(theta: np.ndarray, x: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Analytic gradient of the mean squared error (chain rule, tanh' = 1 - tanh^2)."""
    p = unpack(theta)
    y, (x0, h1, h2) = forward(theta, x)
    n = len(t)
    dy = 2.0 * (y - t) / n                       # (n,)
    g = {}
    g["W3"] = dy[None, :] @ h2                   # (1, 64)
    g["b3"] = np.array([dy.sum()])
    dh2 = dy[:, None] * p["W3"]                  # (n, 64)
    da2 = dh2 * (1.0 - h2 ** 2)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (1.0 - h1 ** 2)
    g["W1"] = da1.T @ x0
    g["b1"] = da1.sum(axis=0)
    return pack(g)


@dataclasses.dataclass
class Adam:
    lr: float
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8

    def run(self, theta: np.ndarray, x: np.ndarray, t: np.ndarray, epochs: int) -> List[float]:
        """Full-batch Adam steps in place; returns the loss before each step."""
        m = np.zeros_like(theta)
        v = np.zeros_like(theta)
        hist = []
        for k in range(1, epochs + 1):
            hist.append(loss(theta, x, t))
            g = grad(theta, x, t)
            m[:] = self.beta1 * m + (1 - self.beta1) * g
            v[:] = self.beta2 * v + (1 - self.beta2) * g * g
            mh = m / (1 - self.beta1 ** k)
            vh = v / (1 - self.beta2 ** k)
            theta -= self.lr * mh / (np.sqrt(vh) + self.eps)
        return hist


def pair_features(C: np.ndarray, r_ops: np.ndarray, pairs, sigma, m_svd, M: int) -> np.ndarray:
    """Eight descriptors per pair [ij] from the localized orbitals C (M x N),
    position operators r_ops (d x M x M) and the pair blocks' singular values:
      d_ij, 1/(1+d_ij), s_i + s_j, |s_i - s_j|, log sigma_1, log sigma_2,
      M_SVD/M, log ||Y^[ij]||_F
    with centroid c_i = (C_i^T r_d C_i)_d, spread s_i = sqrt(sum_d |r_d C_i|^2 - c_id^2)
    and log(x) taken as log(max(x, 1e-300))."""
    cen = np.stack([np.einsum("pi,pq,qi->i", C, r, C) for r in r_ops], axis=1)   # (N, d)
    sq = np.stack([np.sum((r @ C) ** 2, axis=0) for r in r_ops], axis=1)        # (N, d)
    spread = np.sqrt(np.maximum(np.sum(sq - cen ** 2, axis=1), 0.0))
    lg = lambda v: np.log(np.maximum(v, 1e-300))
    rows = []
    for n, (i, j) in enumerate(pairs):
        d = float(np.linalg.norm(cen[i] - cen[j]))
        s = sigma[n]
        rows.append([d, 1.0 / (1.0 + d), spread[i] + spread[j], abs(spread[i] - spread[j]),
                     lg(s[0]), lg(s[1] if len(s) > 1 else 0.0), m_svd[n] / M,
                     0.5 * lg(np.sum(s ** 2))])
    return np.array(rows)


def targets(e_pairs: np.ndarray) -> np.ndarray:
    """log10 of the largest |e_ij(w)| over the training walkers (pairs x walkers in)."""
    return np.log10(np.maximum(np.abs(e_pairs).max(axis=1), 1e-300))
