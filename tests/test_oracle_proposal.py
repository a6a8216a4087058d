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


def test_bf16_rounding_matches_torch():
    """The BF16 rounding of the tensor-core form against torch's conversion
    (round to nearest, ties to even), ties and large values included."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    a = np.concatenate([rng.normal(0, 1, 20000), rng.normal(0, 1e4, 2000),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0, 1e-30])]).astype(np.float32)
    want = torch.tensor(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(PN.bf16(a), want)


def test_bf16_form_reduces_to_the_plain_network_on_representable_values():
    """When every rounded quantity is already a BF16 value (inputs and W1 on
    coarse grids, W2 a signed power-of-two permutation, W3 on a 1/8 grid,
    zero biases in the per-point layers), the BF16 form's forward pass,
    loss and gradient equal the plain network's: the form differs from it by
    the roundings alone."""
    rng = np.random.default_rng(8)
    p = PN.init_params(2)
    W = PN.unflatten(p)
    W[0][:] = rng.integers(-8, 9, W[0].shape) / 8.0
    W[1][:] = 0.0
    W[2][:] = 0.0
    perm = rng.permutation(PN.C2) % PN.C1
    W[2][perm, np.arange(PN.C2)] = rng.choice([-2.0, -1.0, -0.5, 0.5, 1.0, 2.0], PN.C2)
    W[3][:] = 0.0
    W[4][:] = rng.integers(-8, 9, W[4].shape) / 8.0
    W[5][:] = 0.0
    p = np.concatenate([w.ravel() for w in W])
    scans = rng.integers(-8, 9, (2, 16, 3)) / 4.0
    y = np.concatenate([rng.normal(0, 1, (2, 3)), rng.uniform(-np.pi, np.pi, (2, 1)), rng.normal(0, 0.1, (2, 2))], 1)
    f0, f1 = PN.forward(p, scans, 1.0), PN.forward(p, scans, 1.0, bf16_form=True)
    assert np.array_equal(PN.bf16(f0["h1"]), f0["h1"]) and np.array_equal(PN.bf16(f0["h2"]), f0["h2"])
    assert np.allclose(f1["o"], f0["o"], rtol=0, atol=1e-12)
    L0, g0 = PN.loss_grad(p, scans, y, 1.0)
    L1, g1 = PN.loss_grad(p, scans, y, 1.0, bf16_form=True)
    assert abs(L0 - L1) < 1e-12 and np.allclose(g0, g1, rtol=0, atol=1e-12)
    # and a value off the grid does round: the forms then differ
    p2 = p.copy()
    p2[0] += 1e-3
    assert not np.array_equal(PN.forward(p2, scans, 1.0)["h1"], PN.forward(p2, scans, 1.0, bf16_form=True)["h1"])
