"""Learned proposal on the GPU: the sensor simulator against the scene's own
ray casting, the network's forward pass, loss and gradient against the FP64
oracle (oracle/proposal.py), the mixture sampler against the mixture it
samples, and what a trained network gains over uniform seeding."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2404_16370_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def test_simulator_matches_scene_raycast(torch):
    from paper_2404_16370_gb300 import proposal as PR
    room = synth.box_room(1)
    sim = PR.BoxRoomSim(room)
    poses = PR.sample_poses(room, 16, seed=5)
    got = sim.scans(poses, 0.0, seed=1).cpu().numpy().astype(np.float64)
    dirs = synth.fibonacci_sphere(PR.N_POINTS)
    for b, pz in enumerate(poses):
        T = synth.pose_matrix(pz)
        o = np.broadcast_to(T[:3, 3], dirs.shape).copy()
        r = room.raycast(o, dirs @ T[:3, :3].T)
        want = dirs * r[:, None]
        assert np.isfinite(r).all()
        assert np.abs(got[b] - want).max() < 1e-4
    # range noise: zero mean, the requested deviation
    noisy = sim.scans(poses, 0.02, seed=2).cpu().numpy().astype(np.float64)
    dr = np.linalg.norm(noisy, axis=2) * np.sign(np.sum(noisy * dirs, axis=2)) - np.linalg.norm(got, axis=2)
    assert abs(dr.mean()) < 2e-3 and abs(dr.std() - 0.02) < 2e-3


def test_forward_loss_and_gradient_match_oracle(torch):
    from oracle import proposal as PN
    from paper_2404_16370_gb300 import mp, proposal as PR
    B, P = 4, 64
    net = mp.mp_pn_create(P, B, PR.IN_SCALE, PR.SCALE, PR.OFFSET, seed=3)
    try:
        n = mp.mp_pn_num_params(net)
        assert n == PN.NPARAM
        rng = np.random.default_rng(11)
        # random parameters with non-zero biases and a wide last layer
        p = PN.init_params(5)
        p[PN.NPARAM - PN.NOUT - 256 * PN.NOUT:PN.NPARAM - PN.NOUT] *= 20
        k = 0
        for s in PN.SHAPES:
            m = int(np.prod(s))
            if len(s) == 1:
                p[k:k + m] = rng.normal(0, 0.1, m)
            k += m
        mp.mp_pn_set_params(net, torch.tensor(p, dtype=torch.float32, device="cuda"))
        p32 = torch.empty(n, device="cuda")
        mp.mp_pn_get_params(net, p32)
        p64 = p32.cpu().numpy().astype(np.float64)
        scans = rng.normal(0, 3.0, (B, P, 3)).astype(np.float32)
        y = np.concatenate([rng.normal(0, 1, (B, 3)), rng.uniform(-np.pi, np.pi, (B, 1)),
                            rng.normal(0, 0.5, (B, 2))], 1).astype(np.float32)
        xs = torch.tensor(scans, device="cuda")
        ys = torch.tensor(y, device="cuda")
        o = torch.empty((B, mp.MP_PN_OUT), device="cuda")
        mp.mp_pn_forward(net, xs, o)
        loss = torch.zeros(1, device="cuda")
        grad = torch.empty(n, device="cuda")
        mp.mp_pn_loss_grad(net, xs, ys, loss, grad)
        torch.cuda.synchronize()
        ref = PN.forward(p64, scans.astype(np.float64), PR.IN_SCALE)
        L_ref, g_ref = PN.loss_grad(p64, scans.astype(np.float64), y.astype(np.float64), PR.IN_SCALE)
        o_gpu = o.cpu().numpy()
        assert np.abs(o_gpu - ref["o"]).max() <= 1e-4 * max(1.0, np.abs(ref["o"]).max())
        assert abs(float(loss.item()) - L_ref) <= 1e-4 * max(1.0, abs(L_ref))
        g = grad.cpu().numpy()
        # per parameter block: FP32 sums over up to B x P rows
        k = 0
        for s in PN.SHAPES:
            m = int(np.prod(s))
            gb, rb = g[k:k + m], g_ref[k:k + m]
            scale = np.abs(rb).max() + 1e-12
            assert np.abs(gb - rb).max() <= 2e-4 * scale, (s, np.abs(gb - rb).max(), scale)
            k += m
    finally:
        mp.mp_pn_destroy(net)


def test_sampler_follows_the_mixture(torch):
    from paper_2404_16370_gb300 import mp, proposal as PR
    net = mp.mp_pn_create(8, 1, PR.IN_SCALE, PR.SCALE, PR.OFFSET, seed=1)
    try:
        mix = np.zeros(mp.MP_PN_OUT, np.float32)
        mix[:32] = -30.0
        mix[3], mix[17] = np.log(0.25), np.log(0.75)
        means = {3: np.array([1.5, -0.4, 0.1, 2.9, 0.3, -0.2]), 17: np.array([-1.5, 0.6, -0.3, -1.0, -0.4, 0.5])}
        logstd = {3: np.array([-2.0, -1.5, -1.8, -2.5, -1.0, -1.2]), 17: np.array([-1.6, -2.2, -1.4, -2.0, -1.3, -1.1])}
        for c in (3, 17):
            mix[32 + 6 * c:38 + 6 * c] = means[c]
            mix[224 + 6 * c:230 + 6 * c] = 3.0 * np.arctanh(logstd[c] / 3.0)
        n = 400_000
        out = torch.empty((n, 7), device="cuda")
        mp.mp_pn_sample(net, torch.tensor(mix, device="cuda"), n, 42, out)
        poses = out.cpu().numpy().astype(np.float64)
    finally:
        mp.mp_pn_destroy(net)
    ypr = Rotation.from_quat(poses[:, :4]).as_euler("ZYX")
    y = (np.concatenate([poses[:, 4:7], ypr], 1) - PR.OFFSET) / PR.SCALE
    comp17 = y[:, 0] < 0.0            # the components are 7.5 deviations (or more) from x = 0
    assert abs(comp17.mean() - 0.75) < 0.005
    for c, sel in ((3, ~comp17), (17, comp17)):
        d = y[sel] - means[c]
        d[:, 3] = (d[:, 3] + np.pi) % (2 * np.pi) - np.pi
        assert np.all(np.abs(d.mean(0)) < 0.01)
        assert np.all(np.abs(d.std(0) / np.exp(logstd[c]) - 1) < 0.02)


def test_trained_proposal_localises_faster(torch):
    """Train on 50k ray-cast scan/pose pairs (4 epochs), then run 30 seeded
    box-room trials with uniform particles and with 90% of them drawn from
    the network's mixture: the learned seeding localises in fewer steps
    (median) and as often. Both with the preconditioned SVGD reading, with
    which a localised filter stays localised."""
    from paper_2404_16370_gb300 import localise, proposal as PR
    room = synth.box_room(1)
    sim = PR.BoxRoomSim(room)
    poses = PR.sample_poses(room, 50_000, seed=1000)
    scans = sim.scans(poses, 0.02, seed=2000)
    prop = PR.Proposal(128, seed=0)
    try:
        hist = prop.train(scans, PR.targets_of(poses), epochs=4)
        assert hist[-1] < hist[0] - 1.0
        del scans
        _, trials = localise.make_trials(30, 4096, seed0=500)
        q = PR.proposal_quality(prop, sim, trials)
        uni = localise.summarise(localise.run(room, trials, "fp32", 20, svgd_precond=1))
        lrn = localise.summarise(localise.run(room, trials, "fp32", 20, svgd_precond=1,
                                              seeding=PR.seeding_from(prop, sim, trials)))
    finally:
        prop.close()
    print(f"\nproposal: {q}\nuniform: {uni['localised']}/30 median {uni['time_to_localise_median']} steps; "
          f"learned: {lrn['localised']}/30 median {lrn['time_to_localise_median']} steps")
    assert q["trials_with_a_draw_within_tolerance"] > 0.8
    assert lrn["success_rate"] >= uni["success_rate"] - 0.1
    assert lrn["time_to_localise_median"] < uni["time_to_localise_median"]


def bf16_round(a):
    """Round FP32 values to the nearest BF16 (ties to even); returned as float64."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _exact_params(PN, rng):
    """Parameters on a 1/8 grid in [-1, 1]: products with the inputs below are
    exact in BF16 and their sums exact in FP32 up to layer 2."""
    p = np.concatenate([rng.integers(-8, 9, int(np.prod(s))) / 8.0 for s in PN.SHAPES])
    return p.astype(np.float64)


def test_tensor_core_layers_on_exact_inputs(torch):
    """The fused tensor-core kernel (tcgen05 MMAs from 128-byte-swizzled
    shared memory, accumulators in TMEM, max-pool in the epilogue) against a
    float64 evaluation of the same BF16 network: inputs on a 1/4 grid and
    weights on a 1/8 grid make layer 1 and layer 2 exact in both, layer 2's
    BF16 rounding is reproduced in numpy, and only layer 3's FP32 summation
    order differs. A wrong operand layout, swizzle or descriptor would move
    the outputs by O(1)."""
    from oracle import proposal as PN
    from paper_2404_16370_gb300 import mp, proposal as PR
    B, P = 3, 384
    net = mp.mp_pn_create(P, B, 1.0, PR.SCALE, PR.OFFSET, seed=3)
    try:
        rng = np.random.default_rng(17)
        p = _exact_params(PN, rng)
        mp.mp_pn_set_params(net, torch.tensor(p, dtype=torch.float32, device="cuda"))
        scans = (rng.integers(-8, 9, (B, P, 3)) / 4.0).astype(np.float32)
        o = torch.empty((B, mp.MP_PN_OUT), device="cuda")
        mp.mp_pn_forward(net, torch.tensor(scans, device="cuda"), o)
        mp.mp_pn_status(net)
        o_tc = o.cpu().numpy().astype(np.float64)
        W1, b1, W2, b2, W3, b3, W4, b4, W5, b5 = PN.unflatten(p)
        x = scans.astype(np.float64)
        h1 = np.maximum(x @ W1 + b1, 0.0)
        assert np.array_equal(bf16_round(h1), h1)            # layer 1 exact in BF16
        h2 = np.maximum(h1 @ W2 + b2, 0.0)                   # exact in FP32 accumulation
        h3 = np.maximum(bf16_round(h2) @ W3 + b3, 0.0)
        g = h3.max(axis=1)
        o_ref = np.maximum(g @ W4 + b4, 0.0) @ W5 + b5
        assert np.abs(o_tc - o_ref).max() <= 1e-5 * np.abs(o_ref).max(), np.abs(o_tc - o_ref).max()
        # the CUDA-core FP32 path on the same parameters: layer 2 unrounded
        mp.mp_pn_set_precision(net, mp.MP_PREC_FP32)
        mp.mp_pn_forward(net, torch.tensor(scans, device="cuda"), o)
        o32 = o.cpu().numpy().astype(np.float64)
        g32 = np.maximum(h2 @ W3 + b3, 0.0).max(axis=1)
        o32_ref = np.maximum(g32 @ W4 + b4, 0.0) @ W5 + b5
        assert np.abs(o32 - o32_ref).max() <= 1e-5 * np.abs(o32_ref).max()
    finally:
        mp.mp_pn_destroy(net)


def test_tensor_core_forward_and_gradient_against_oracle(torch):
    """The BF16 tensor-core form of the per-point layers (FP32 master weights
    and backward pass) against the oracle: element by element against the
    oracle's BF16 form of the network (the same roundings; FP32 against FP64
    sums), and against the plain FP64 network within the BF16 tolerance
    stated here (outputs and loss 2e-2 of their scale; gradient blocks 0.25
    in relative norm, where a BF16 rounding that moves a channel's max-pool to
    another point moves that channel's whole gradient path); and the BF16
    form beats the FP32 CUDA-core form on a training-size batch."""
    import time
    from oracle import proposal as PN
    from paper_2404_16370_gb300 import mp, proposal as PR
    B, P = 4, 256
    net = mp.mp_pn_create(P, B, PR.IN_SCALE, PR.SCALE, PR.OFFSET, seed=3)
    try:
        n = mp.mp_pn_num_params(net)
        rng = np.random.default_rng(11)
        p = PN.init_params(5)
        k = 0
        for s in PN.SHAPES:
            m = int(np.prod(s))
            if len(s) == 1:
                p[k:k + m] = rng.normal(0, 0.1, m)
            k += m
        mp.mp_pn_set_params(net, torch.tensor(p, dtype=torch.float32, device="cuda"))
        p32 = torch.empty(n, device="cuda")
        mp.mp_pn_get_params(net, p32)
        p64 = p32.cpu().numpy().astype(np.float64)
        scans = rng.normal(0, 3.0, (B, P, 3)).astype(np.float32)
        y = np.concatenate([rng.normal(0, 1, (B, 3)), rng.uniform(-np.pi, np.pi, (B, 1)),
                            rng.normal(0, 0.5, (B, 2))], 1).astype(np.float32)
        xs, ys = torch.tensor(scans, device="cuda"), torch.tensor(y, device="cuda")
        o = torch.empty((B, mp.MP_PN_OUT), device="cuda")
        mp.mp_pn_forward(net, xs, o)
        loss = torch.zeros(1, device="cuda")
        grad = torch.empty(n, device="cuda")
        mp.mp_pn_loss_grad(net, xs, ys, loss, grad)
        mp.mp_pn_status(net)
        o_gpu, g = o.cpu().numpy(), grad.cpu().numpy()
        s64, y64 = scans.astype(np.float64), y.astype(np.float64)
        for form, o_tol, g_tol in ((True, 1e-5, 1e-5), (False, 2e-2, 0.25)):
            ref = PN.forward(p64, s64, PR.IN_SCALE, bf16_form=form)
            L_ref, g_ref = PN.loss_grad(p64, s64, y64, PR.IN_SCALE, bf16_form=form)
            name = "BF16 form" if form else "plain FP64"
            err_o = np.abs(o_gpu - ref["o"]).max() / max(1.0, np.abs(ref["o"]).max())
            print(f"\n{name}: outputs {err_o:.2e}, loss {abs(float(loss.item()) - L_ref):.2e}")
            assert err_o <= o_tol
            assert abs(float(loss.item()) - L_ref) <= o_tol * max(1.0, abs(L_ref))
            k = 0
            for s in PN.SHAPES:
                m = int(np.prod(s))
                gb, rb = g[k:k + m], g_ref[k:k + m]
                rel = np.linalg.norm(gb - rb) / (np.linalg.norm(rb) + 1e-12)
                print(f"{name}: gradient block {s}: relative error {rel:.2e}")
                assert rel <= g_tol, (name, s, rel)
                k += m
    finally:
        mp.mp_pn_destroy(net)
    # speed on a training-size batch: 128 scans of 1024 points
    B, P = 128, 1024
    net = mp.mp_pn_create(P, B, PR.IN_SCALE, PR.SCALE, PR.OFFSET, seed=3)
    try:
        xs = torch.tensor(rng.normal(0, 3.0, (B, P, 3)).astype(np.float32), device="cuda")
        o = torch.empty((B, mp.MP_PN_OUT), device="cuda")
        ms = {}
        for prec in (mp.MP_PREC_FP32, mp.MP_PREC_BF16):
            mp.mp_pn_set_precision(net, prec)
            for _ in range(3):
                mp.mp_pn_forward(net, xs, o)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(20):
                mp.mp_pn_forward(net, xs, o)
            torch.cuda.synchronize()
            ms[prec] = (time.perf_counter() - t0) / 20 * 1e3
        mp.mp_pn_status(net)
        print(f"forward of 128 x 1024 points: FP32 CUDA cores {ms[mp.MP_PREC_FP32]:.3f} ms, "
              f"BF16 tensor cores {ms[mp.MP_PREC_BF16]:.3f} ms")
        assert ms[mp.MP_PREC_BF16] < ms[mp.MP_PREC_FP32]
    finally:
        mp.mp_pn_destroy(net)
