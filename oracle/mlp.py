"""Oracle of the sigma policy network -- TEST INFRASTRUCTURE ONLY (tests, smoke check).

Plain numpy in FP64: the forward pass of the 64-64-64-64-5 ReLU network, the regression
loss L = mean_i 1/2 (q(x_i)[a_i] - y_i)^2 and its gradient by the chain rule, written
layer by layer.  With `bf16=True` the weights are first rounded to BF16 (round to
nearest, ties to even, on the FP32 bit pattern), as the CUDA kernels use them; the
gradient is then the gradient with respect to those rounded weights.  ReLU'(0) = 0.
Shares no code with the CUDA path.

Parameter layout: W1 (64x64), b1, W2 (64x64), b2, W3 (64x64), b3, W4 (5x64), b4, each W
row-major [out][in].
"""
import numpy as np

IN, H, OUT = 64, 64, 5
SHAPES = [(H, IN), (H,), (H, H), (H,), (H, H), (H,), (OUT, H), (OUT,)]
P = sum(int(np.prod(s)) for s in SHAPES)


def bf16_round(w):
    """FP32 -> BF16 (kept in float64): round the FP32 bits to the upper 16, nearest-even."""
    f = np.ascontiguousarray(w, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(w):
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(np.asarray(w[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1) for p in parts])


def forward(w, X, bf16=True):
    """q (n x 5) and the pre-activations (z1, z2, z3)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(bf16_round(w) if bf16 else np.asarray(w, np.float64))
    X = np.asarray(X, np.float64).reshape(-1, IN)
    z1 = X @ W1.T + b1
    z2 = np.maximum(z1, 0.0) @ W2.T + b2
    z3 = np.maximum(z2, 0.0) @ W3.T + b3
    q = np.maximum(z3, 0.0) @ W4.T + b4
    return q, (z1, z2, z3)


def loss_grad(w, X, act, y, bf16=True):
    """(L, dL/dw) for L = mean_i 1/2 (q_i[a_i] - y_i)^2."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(bf16_round(w) if bf16 else np.asarray(w, np.float64))
    X = np.asarray(X, np.float64).reshape(-1, IN)
    act = np.asarray(act, np.int64)
    y = np.asarray(y, np.float64)
    n = X.shape[0]
    q, (z1, z2, z3) = forward(w, X, bf16)
    e = q[np.arange(n), act] - y
    L = 0.5 * np.mean(e * e)
    dq = np.zeros_like(q)
    dq[np.arange(n), act] = e / n
    a1, a2, a3 = np.maximum(z1, 0.0), np.maximum(z2, 0.0), np.maximum(z3, 0.0)
    gW4 = dq.T @ a3
    gb4 = dq.sum(0)
    d3 = (dq @ W4) * (z3 > 0)
    gW3 = d3.T @ a2
    gb3 = d3.sum(0)
    d2 = (d3 @ W3) * (z2 > 0)
    gW2 = d2.T @ a1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (z1 > 0)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    return L, pack([gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4])


def init(seed):
    """He-style initial weights (normal, std sqrt(2 / fan_in)), zero biases, as FP32."""
    rng = np.random.default_rng([0x5167, seed])
    parts = []
    for s in SHAPES:
        parts.append(rng.standard_normal(s) * np.sqrt(2.0 / s[1]) if len(s) == 2 else np.zeros(s))
    return pack(parts).astype(np.float32)
