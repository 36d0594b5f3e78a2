"""The sigma policy network's CUDA kernels against the numpy oracle (oracle/mlp.py):
forward outputs, loss and gradient with the same BF16-rounded weights (FP32 accumulation
on the GPU, FP64 in the oracle), and training that lowers the loss."""
import numpy as np
import pytest

from paper_2408_12179_b300 import hpr

pytestmark = pytest.mark.gpu

from oracle import mlp


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hpr.load()


def _data(seed, n):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((n, 64)) * 0.5).astype(np.float32)
    return X, rng.integers(0, 5, n).astype(np.int32), rng.standard_normal(n).astype(np.float32)


def test_param_count():
    assert hpr.mlp_param_count() == mlp.P == 12805


def test_infer_matches_oracle():
    X, _, _ = _data(1, 257)
    w = mlp.init(7)
    Q = hpr.mlp_infer(w, X)
    ref, _ = mlp.forward(w, X.astype(np.float64), bf16=True)
    assert np.linalg.norm(Q - ref) / np.linalg.norm(ref) <= 1e-5


@pytest.mark.parametrize("n", [1, 300, 2000])
def test_gradient_matches_oracle(n):
    X, a, y = _data(2, n)
    w = mlp.init(8)
    L, g = hpr.mlp_grad(w, X, a, y)
    Lr, gr = mlp.loss_grad(w, X.astype(np.float64), a, y.astype(np.float64), bf16=True)
    assert L == pytest.approx(Lr, rel=1e-5)
    offs = np.cumsum([0] + [int(np.prod(s)) for s in mlp.SHAPES])
    for i in range(len(mlp.SHAPES)):              # every layer's block on its own
        gi, ri = g[offs[i]:offs[i + 1]], gr[offs[i]:offs[i + 1]]
        assert np.linalg.norm(gi - ri) <= 1e-4 * max(np.linalg.norm(ri), 1e-12), (i, n)


def test_training_lowers_the_loss():
    """A teacher network labels random inputs; training a fresh network on them for 40
    passes lowers the loss at least tenfold, deterministically."""
    X, a, _ = _data(3, 4096)
    teacher = mlp.init(11)
    y = mlp.forward(teacher, X.astype(np.float64), bf16=True)[0][np.arange(len(a)), a].astype(np.float32)
    w0 = mlp.init(12)
    L0 = mlp.loss_grad(w0, X.astype(np.float64), a, y.astype(np.float64))[0]
    w1, hist = hpr.mlp_train(w0, X, a, y, epochs=40, batch=256, lr=2e-3, seed=5)
    w2, hist2 = hpr.mlp_train(w0, X, a, y, epochs=40, batch=256, lr=2e-3, seed=5)
    assert np.array_equal(w1, w2) and np.array_equal(hist, hist2)
    L1 = mlp.loss_grad(w1, X.astype(np.float64), a, y.astype(np.float64))[0]
    print(f"loss {L0:.4f} -> {L1:.5f}; per-epoch {hist[0]:.4f} ... {hist[-1]:.5f}")
    assert L1 <= 0.1 * L0
    assert hist[-1] < hist[0]


def test_policy_in_the_solver():
    """Exploring solves yield samples; a network trained on them drives sigma at restarts
    (sigma_policy 2); the solve still converges with an independently checked KKT, every
    restart is either a learned decision or a counted fallback, and exploration draws
    multipliers 2^((a-2)/2) of Algorithm 3's sigma."""
    from paper_2408_12179_b300 import lpgen, policy
    from oracle import kkt as K

    train = [lpgen.planted_medium(1, 0.005), lpgen.mcf_lp(2, nodes=100)]
    X, A, Y = policy.collect(train, seeds=(3,))
    assert len(Y) > 10 and set(A.tolist()) <= set(range(5)) and np.all(np.isfinite(Y))
    with hpr.Solver(train[0], sigma_policy=1, policy_seed=3) as s:
        s.solve(1e-8)
        for r in s.checks():
            if r["action"] >= 0:
                assert r["sigma_next"] == pytest.approx(r["sigma_rule"] * 2.0 ** ((r["action"] - 2) / 2), rel=1e-15)
    w, hist = policy.train(X, A, Y, epochs=30)
    assert hist[-1] < hist[0]
    lp = lpgen.planted_medium(7, 0.005)
    rows = policy.evaluate([lp], w)
    r = rows[0]
    assert r["rule_status"] == hpr.HPR_OK and r["policy_status"] == hpr.HPR_OK
    assert r["decisions"] > 0
    with hpr.Solver(lp, sigma_policy=2) as s:
        s.set_policy(w)
        res = s.solve(1e-8)
        restarts = sum(1 for c in s.checks() if c["cause"] > 0)
    ind = K.kkt(lp, res["x"], res["y"], res["z"])
    assert ind["kkt"] <= 1e-8 * (1 + 1e-6)
    I = res["info"]
    assert I["policy_decisions"] + I["policy_fallbacks"] <= restarts
    print(f"iterations: rule {r['rule_iters']}, policy {r['policy_iters']} "
          f"({r['decisions']} decisions, {r['fallbacks']} fallbacks)")
