"""Pins for the scheduler's CPU reference: gradient against central finite
differences of the loss, and closed forms of the forward pass."""
import numpy as np

from oracle import sched_ref as R


def _rand(seed, n=40):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.4, R.COUNT)
    p[:5] = rng.normal(0, 1, 5)          # mu
    p[5:10] = rng.uniform(0.5, 1.5, 5)   # isd
    x = rng.normal(0, 2, (n, 5))
    y = rng.normal(0, 1, (n, 3))
    return p, x, y


def test_gradient_matches_finite_differences():
    for seed in range(3):
        p, x, y = _rand(seed)
        g = R.grad(p, x, y)
        h = 1e-6
        rng = np.random.default_rng(seed)
        for i in list(range(10)) + list(rng.choice(R.COUNT, 200, replace=False)):
            d = np.zeros(R.COUNT)
            d[i] = h
            fd = (R.loss(p + d, x, y) - R.loss(p - d, x, y)) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_forward_closed_forms():
    p, x, _ = _rand(7)
    q = p.copy()
    P = R.unpack(q)
    P["W3"][:] = 0.0  # outputs reduce to the output bias
    o, _ = R.forward(q, x)
    assert np.allclose(o, P["b3"])
    q = p.copy()
    P = R.unpack(q)
    P["W1"][:] = 0.0
    P["b1"][:] = -1.0  # first layer dead: outputs = W3 relu(b2) + b3
    o, _ = R.forward(q, x)
    assert np.allclose(o, P["W3"] @ np.maximum(P["b2"], 0) + P["b3"])
    assert R.COUNT == 1357


def test_loss_is_mean_square():
    p, x, y = _rand(3, n=7)
    o, _ = R.forward(p, x)
    assert np.isclose(R.loss(p, x, y), ((o - y) ** 2).mean())


def test_host_feature_function_matches_reference():
    """truss_sched_features (host code in the library) computes the
    reference features; no GPU call is made."""
    import __graft_entry__

    __graft_entry__.build()
    import paper_1707_02000_gb300 as pkt

    tr = np.zeros(6, pkt.TRACE_DTYPE)
    tr["level"] = [0, 1, 5, 20, 100, 900]
    tr["n_light"] = [0, 3, 100, 1000, 5, 123456]
    tr["n_heavy"] = [1, 0, 7, 9999, 5, 2]
    tr["dsum"] = [40, 3, 2000, 10 ** 9, 77, 3]
    tr["dmax"] = [40, 1, 60, 12000, 9, 1]
    tr["todo"] = [10, 3, 10 ** 7, 2 * 10 ** 8, 12, 123458]
    x = pkt.sched_features(tr)
    want = R.features(tr["n_light"] + tr["n_heavy"], tr["dsum"], tr["dmax"], tr["level"], tr["todo"])
    assert np.allclose(x, want, rtol=1e-6, atol=1e-6)
