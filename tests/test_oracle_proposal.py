"""Pins of the FP64 proposal-network oracle (CPU): its gradient against central
finite differences of its loss, its mixture likelihood against a closed form
and the periodicity of the yaw dimension."""
import numpy as np
import pytest
from scipy.stats import norm

from oracle import proposal as PN


def small_case(seed=1, B=3, P=24):
    rng = np.random.default_rng(seed)
    p = PN.init_params(seed)
    # non-zero biases and a larger last layer so that every term is exercised
    k = 0
    for s in PN.SHAPES:
        n = int(np.prod(s))
        if len(s) == 1:
            p[k:k + n] = rng.normal(0, 0.1, n)
        k += n
    p[-PN.NOUT - PN.C4 * PN.NOUT:-PN.NOUT] *= 20
    scans = rng.normal(0, 3.0, (B, P, 3))
    y = np.concatenate([rng.normal(0, 1, (B, 3)), rng.uniform(-np.pi, np.pi, (B, 1)), rng.normal(0, 0.1, (B, 2))], 1)
    return p, scans, y


def test_parameter_layout():
    assert PN.NPARAM == 3 * 64 + 64 + 64 * 128 + 128 + 128 * 256 + 256 + 256 * 256 + 256 + 256 * 416 + 416


def test_gradient_matches_finite_differences():
    p, scans, y = small_case()
    L, g = PN.loss_grad(p, scans, y, 5.0)
    assert abs(L - PN.loss(p, scans, y, 5.0)) < 1e-12
    rng = np.random.default_rng(7)
    # every block: a random subset of its entries
    idx, k = [], 0
    for s in PN.SHAPES:
        n = int(np.prod(s))
        idx += list(k + rng.choice(n, min(n, 24), replace=False))
        k += n
    h = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += h
        lp = PN.loss(q, scans, y, 5.0)
        q[i] -= 2 * h
        lm = PN.loss(q, scans, y, 5.0)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_single_component_is_a_diagonal_gaussian():
    rng = np.random.default_rng(3)
    o = rng.normal(0, 0.3, (4, PN.NOUT))
    o[:, 0] = 60.0                      # component 0 carries all the weight
    y = rng.normal(0, 0.5, (4, 6))
    m = o[:, 32:38]
    s = 3.0 * np.tanh(o[:, 224:230] / 3.0)
    want = -np.sum(norm.logpdf(y, loc=m, scale=np.exp(s)), axis=1)
    assert np.allclose(PN.nll(o, y), want, rtol=0, atol=1e-9)


def test_yaw_is_periodic():
    rng = np.random.default_rng(4)
    o = rng.normal(0, 0.5, (5, PN.NOUT))
    y = rng.normal(0, 0.5, (5, 6))
    y2 = y.copy()
    y2[:, 3] += 2 * np.pi
    y3 = y.copy()
    y3[:, 3] -= 4 * np.pi
    assert np.allclose(PN.nll(o, y), PN.nll(o, y2), atol=1e-9)
    assert np.allclose(PN.nll(o, y), PN.nll(o, y3), atol=1e-9)


@pytest.mark.parametrize("B", [1, 2])
def test_maxpool_routes_to_the_first_maximum(B):
    p, scans, y = small_case(seed=5, B=B, P=4)
    scans[:, 1] = scans[:, 0]           # duplicate points: ties in every channel
    f = PN.forward(p, scans, 5.0)
    assert np.all(f["gi"] != 1)         # the tie goes to the first point
    _, g = PN.loss_grad(p, scans, y, 5.0)
    assert np.all(np.isfinite(g))
