"""FP64 reference of the beam/stop network: forward pass, loss and
back-propagated gradient.  TEST INFRASTRUCTURE ONLY (tests and smoke check).

Network (the learned search policy): 12 input features -> 64 ReLU -> 64 ReLU
-> nl + 1 outputs: nl logits over the beam ladder and one stop-hop output.
Loss: mean cross-entropy of the logits against the beam class y plus
lam * mean squared error of the stop output against t.
Parameters are one flat vector: W1 [64][12], b1 [64], W2 [64][64], b2 [64],
W3 [nl+1][64], b3 [nl+1] (row-major, output by input).
"""
import numpy as np

NFEAT = 12
HID = 64


def n_params(nl):
    return HID * NFEAT + HID + HID * HID + HID + (nl + 1) * HID + (nl + 1)


def unpack(theta, nl):
    theta = np.asarray(theta, np.float64)
    shapes = [("W1", (HID, NFEAT)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
              ("W3", (nl + 1, HID)), ("b3", (nl + 1,))]
    out, off = {}, 0
    for name, shp in shapes:
        size = int(np.prod(shp))
        out[name] = theta[off:off + size].reshape(shp)
        off += size
    assert off == theta.size
    return out


def forward(theta, X, nl):
    p = unpack(theta, nl)
    X = np.asarray(X, np.float64)
    A1 = X @ p["W1"].T + p["b1"]
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ p["W2"].T + p["b2"]
    H2 = np.maximum(A2, 0.0)
    Z = H2 @ p["W3"].T + p["b3"]
    return Z, (X, A1, H1, A2, H2)


def loss(theta, X, y, t, nl, lam):
    Z, _ = forward(theta, X, nl)
    logits = Z[:, :nl]
    m = logits.max(axis=1, keepdims=True)
    lse = (m[:, 0] + np.log(np.exp(logits - m).sum(axis=1)))
    ce = np.mean(lse - logits[np.arange(len(y)), y])
    mse = np.mean((Z[:, nl] - np.asarray(t, np.float64)) ** 2)
    return ce + lam * mse


def grad(theta, X, y, t, nl, lam):
    """d loss / d theta by back-propagation, flat like theta."""
    p = unpack(theta, nl)
    Z, (X, A1, H1, A2, H2) = forward(theta, X, nl)
    B = X.shape[0]
    logits = Z[:, :nl]
    e = np.exp(logits - logits.max(axis=1, keepdims=True))
    soft = e / e.sum(axis=1, keepdims=True)
    dZ = np.zeros_like(Z)
    dZ[:, :nl] = soft
    dZ[np.arange(B), y] -= 1.0
    dZ[:, :nl] /= B
    dZ[:, nl] = 2.0 * lam * (Z[:, nl] - np.asarray(t, np.float64)) / B
    gW3 = dZ.T @ H2
    gb3 = dZ.sum(axis=0)
    dH2 = dZ @ p["W3"]
    dA2 = dH2 * (A2 > 0)
    gW2 = dA2.T @ H1
    gb2 = dA2.sum(axis=0)
    dH1 = dA2 @ p["W2"]
    dA1 = dH1 * (A1 > 0)
    gW1 = dA1.T @ X
    gb1 = dA1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def init_params(nl, seed=0):
    """He-style initial weights (zero biases) from a seeded generator."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.standard_normal((HID, NFEAT)) * np.sqrt(2.0 / NFEAT), np.zeros(HID),
             rng.standard_normal((HID, HID)) * np.sqrt(2.0 / HID), np.zeros(HID),
             rng.standard_normal((nl + 1, HID)) * np.sqrt(1.0 / HID), np.zeros(nl + 1)]
    return np.concatenate([q.ravel() for q in parts])
