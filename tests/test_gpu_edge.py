"""Edge cases, error returns and the failure path of the CUDA library, through
the C ABI: a single particle, ragged sizes (particles and scan points not
multiples of the block/chunk sizes), a scan whose points are all invalid, the
largest scan, a blackout step (empty scan), device-pointer inputs on a caller
stream, invalid arguments, and bounded device waits made to give up (test
knobs withhold 16 announced bytes of a bulk copy, or make a grid barrier wait
for one CTA more than the grid has; nothing faults or hangs)."""
import numpy as np
import pytest

from gpu_util import check_sums
from paper_2404_16370_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def room(oracle):
    w = synth.box_room_workload(n_particles=8192)
    P = oracle.Params.box_room(4096)
    return dict(w=w, om=oracle.OracleMap(w.map_points, P), P=P)


def make_ctx(mp, room, n, **over):
    params = mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, n, **over)
    ctx = mp.mp_init_map(room["w"].map_points, params)
    mp.mp_init_particles(ctx, n, poses=room["w"].particles[:n])
    return ctx


def test_single_particle(room):
    from paper_2404_16370_gb300 import mp
    ctx = make_ctx(mp, room, 1)
    try:
        mp.mp_step(ctx, room["w"].scans[0])
        best, bp = mp.mp_get_posterior(ctx)
        ids = mp.mp_get_buffer(ctx, mp.MP_BUF_NBR_IDS)
        post = mp.mp_get_buffer(ctx, mp.MP_BUF_POST)
        poses = mp.mp_get_buffer(ctx, mp.MP_BUF_POSES)
    finally:
        mp.mp_destroy(ctx)
    assert post.tolist() == [1.0] and bp == 1.0
    assert ids[0, 0] == 0 and np.all(ids[0, 1:] == -1)
    assert np.array_equal(best, poses[0])


@pytest.mark.parametrize("n,npts", [(4099, 300), (129, 257), (3, 1)])
def test_ragged_likelihood(room, oracle, n, npts):
    from paper_2404_16370_gb300 import mp
    sc = room["w"].scans[0][:npts]
    ctx = make_ctx(mp, room, n)
    try:
        mp.mp_set_scan(ctx, sc)
        mp.mp_run_stages(ctx, mp.MP_STAGE_SCAN | mp.MP_STAGE_LIKELIHOOD)
        gn = mp.mp_get_buffer(ctx, mp.MP_BUF_GN)
    finally:
        mp.mp_destroy(ctx)
    P = room["P"]
    sn, sv, _, _ = oracle.point_normals(sc, P.r_cov, P.cov_k, P.cov_min)
    ref = oracle.likelihood(room["om"], room["w"].particles[:n], sc, sn, sv, P, amb_tol=1e-4)
    msg = check_sums(gn, ref)
    assert not msg, msg


def test_all_scan_points_invalid(room):
    from paper_2404_16370_gb300 import mp
    sc = np.array([[0, 0, 0], [10, 0, 0], [0, 10, 0], [0, 0, 10]], np.float32)   # no neighbours within r_cov
    ctx = make_ctx(mp, room, 100)
    try:
        mp.mp_step(ctx, sc)
        gn = mp.mp_get_buffer(ctx, mp.MP_BUF_GN)
        psi = mp.mp_get_buffer(ctx, mp.MP_BUF_PSI)
        valid = mp.mp_get_buffer(ctx, mp.MP_BUF_SCAN_VALID)
        post = mp.mp_get_buffer(ctx, mp.MP_BUF_POST)
    finally:
        mp.mp_destroy(ctx)
    assert not valid.any()
    assert np.all(gn == 0) and np.all(psi == 0)
    assert abs(post.sum() - 1) < 1e-12 and np.allclose(post, 1 / 100, rtol=1e-12)


def test_largest_scan_and_limit(room):
    from paper_2404_16370_gb300 import mp
    dirs = synth.spherical_dirs(1024)
    sc = synth.scan(room["w"].scene, room["w"].gt[0], dirs, 0.02, 9)
    assert len(sc) == 1024
    ctx = make_ctx(mp, room, 256, max_scan=1024)
    try:
        mp.mp_step(ctx, sc)
        mp.mp_get_posterior(ctx)
        with pytest.raises(mp.MPError) as e:
            mp.mp_step(ctx, np.concatenate([sc, sc[:1]]))
        assert e.value.code == mp.MP_EINVAL
    finally:
        mp.mp_destroy(ctx)


def test_blackout_step_matches_oracle(room, oracle):
    from paper_2404_16370_gb300 import mp
    n = 2048
    P = oracle.Params.box_room(n)
    rng = np.random.default_rng(3)
    logprior = -rng.uniform(0, 30, n)
    ctx = make_ctx(mp, room, n)
    try:
        mp.mp_set_buffer(ctx, mp.MP_BUF_LOG_PRIOR, logprior)
        mp.mp_step(ctx, None)                     # empty scan, identity odometry, no noise
        post = mp.mp_get_buffer(ctx, mp.MP_BUF_POST)
        ids = mp.mp_get_buffer(ctx, mp.MP_BUF_NBR_IDS)
        poses = mp.mp_get_buffer(ctx, mp.MP_BUF_POSES)
    finally:
        mp.mp_destroy(ctx)
    f = oracle.OracleFilter(room["om"], P, room["w"].particles[:n].copy(), logprior=logprior.copy())
    out = f.step(np.zeros((0, 3), np.float32))
    assert np.array_equal(poses, room["w"].particles[:n])       # no correction in a blackout
    ok = out["merge_flags"] == 0
    same = np.array([set(a[a >= 0]) == set(b[b >= 0]) for a, b in zip(ids, out["nbr_ids"])])
    assert same[ok].all()
    good = ok.copy()
    for i in np.nonzero(~ok)[0]:               # a flagged list changes its neighbours' smoothing
        good[out["nbr_ids"][i][out["nbr_ids"][i] >= 0]] = False
    assert np.allclose(post[good], out["post"][good], rtol=1e-5, atol=1e-300)
    assert abs(post.sum() - 1) < 1e-12


def test_device_inputs_on_caller_stream(room):
    import torch
    from paper_2404_16370_gb300 import mp
    n = 1024
    sc = room["w"].scans[0]
    outs = []
    for use_dev in (False, True):
        stream = torch.cuda.Stream()
        params = mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, n)
        ctx = mp.mp_init_map(room["w"].map_points, params, cuda_stream=stream.cuda_stream)
        try:
            if use_dev:
                poses = torch.from_numpy(room["w"].particles[:n]).cuda()
                mp.mp_init_particles(ctx, n, poses=poses)
                mp.mp_step(ctx, torch.from_numpy(sc).cuda())
            else:
                mp.mp_init_particles(ctx, n, poses=room["w"].particles[:n])
                mp.mp_step(ctx, sc)
            gn = torch.empty((n, 29), dtype=torch.float32, device="cuda")
            mp.mp_get_buffer(ctx, mp.MP_BUF_GN, out=gn)
            outs.append(gn.cpu().numpy())
        finally:
            mp.mp_destroy(ctx)
    assert np.array_equal(outs[0], outs[1])


def test_merge_after_keys_without_sort(room):
    """Stages out of order: fresh LSH buckets with the segment table of no
    sort (never written after the particles' initialisation). The merge's
    window is empty wherever the table does not hold the particle, so the
    lists keep only valid ids (self and the previous list)."""
    from paper_2404_16370_gb300 import mp
    n = 2048
    ctx = make_ctx(mp, room, n)
    try:
        mp.mp_set_step_index(ctx, 3)
        mp.mp_run_stages(ctx, mp.MP_STAGE_LSH)
        mp.mp_run_stages(ctx, mp.MP_STAGE_MERGE)
        ids = mp.mp_get_buffer(ctx, mp.MP_BUF_NBR_IDS)
    finally:
        mp.mp_destroy(ctx)
    assert ids.min() >= -1 and ids.max() < n
    assert np.array_equal(ids[:, 0], np.arange(n))   # self first


def test_invalid_arguments(room):
    from paper_2404_16370_gb300 import mp
    with pytest.raises(mp.MPError):
        mp.mp_init_map(room["w"].map_points, mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, 64, K=33))
    with pytest.raises(mp.MPError):
        mp.mp_init_map(room["w"].map_points, mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, 64, nnf_res=0.0))
    ctx = mp.mp_init_map(room["w"].map_points, mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, 64))
    try:
        with pytest.raises(mp.MPError) as e:
            mp.mp_step(ctx, room["w"].scans[0])
        assert e.value.code == mp.MP_ENOTINIT
        with pytest.raises(mp.MPError) as e:
            mp.mp_init_particles(ctx, 0, poses=room["w"].particles[:1])
        assert e.value.code == mp.MP_EINVAL
        mp.mp_init_particles(ctx, 64, poses=room["w"].particles[:64])
        L = mp.lib()
        assert L.mp_step(ctx, None, 5, None, None) == mp.MP_EINVAL          # NULL scan with n_scan > 0
        assert L.mp_step(ctx, None, -1, None, None) == mp.MP_EINVAL
        with pytest.raises(mp.MPError) as e:
            mp.mp_get_buffer(ctx, mp.MP_BUF_POSES, out=np.zeros((63, 7), np.float32))
        assert e.value.code == mp.MP_EINVAL
        with pytest.raises(mp.MPError):
            mp.mp_set_buffer(ctx, mp.MP_BUF_KEYS, np.zeros(64, np.uint32))   # read-only buffer
        with pytest.raises(mp.MPError):
            mp.mp_set_buffer(ctx, mp.MP_BUF_VISIT_ORDER, np.zeros(64, np.int32))   # not a permutation
        mp.mp_set_buffer(ctx, mp.MP_BUF_VISIT_ORDER, np.arange(64, dtype=np.int32)[::-1].copy())
        assert np.array_equal(mp.mp_get_buffer(ctx, mp.MP_BUF_VISIT_ORDER), np.arange(64)[::-1])
        # index buffers the kernels gather through are checked before upload
        dup = np.arange(64, dtype=np.int32)
        dup[5] = 4
        with pytest.raises(mp.MPError) as e:
            mp.mp_set_buffer(ctx, mp.MP_BUF_SORTED_IDS, dup)
        assert "permutation" in mp.mp_last_error(ctx)
        K = mp.mp_buffer_size(ctx, mp.MP_BUF_NBR_IDS) // 64
        ids = np.full((64, K), -1, np.int32)
        ids[3, 1] = 64
        with pytest.raises(mp.MPError) as e:
            mp.mp_set_buffer(ctx, mp.MP_BUF_NBR_IDS, ids)
        assert "[-1, n)" in mp.mp_last_error(ctx)
        mp.mp_set_buffer(ctx, mp.MP_BUF_SORTED_IDS, np.arange(64, dtype=np.int32)[::-1].copy())
        assert np.array_equal(mp.mp_get_buffer(ctx, mp.MP_BUF_SORTED_IDS), np.arange(64)[::-1])
        bad = np.eye(4)
        bad[0, 3] = np.nan
        with pytest.raises(mp.MPError):
            mp.mp_set_odometry(ctx, bad)
        assert "not finite" in mp.mp_last_error(ctx)
    finally:
        mp.mp_destroy(ctx)


def test_bounded_wait_gives_up_and_context_recovers(room, oracle):
    """A barrier that never completes (16 announced bytes never arrive): the
    likelihood kernel's bounded wait gives up after ~1 ms of SM clock, records
    the error and returns; the host sees MP_ETIMEOUT; the next run is normal."""
    from paper_2404_16370_gb300 import mp
    n = 512
    sc = room["w"].scans[0]
    ctx = make_ctx(mp, room, n)
    try:
        mp.mp_debug_set(ctx, mp.MP_DEBUG_WAIT_BUDGET, 2_000_000)
        mp.mp_debug_set(ctx, mp.MP_DEBUG_STARVE_TX, 1)
        mp.mp_set_scan(ctx, sc)
        mp.mp_run_stages(ctx, mp.MP_STAGE_SCAN | mp.MP_STAGE_LIKELIHOOD)
        with pytest.raises(mp.MPError) as e:
            mp.mp_get_posterior(ctx)
        assert e.value.code == mp.MP_ETIMEOUT
        mp.mp_debug_set(ctx, mp.MP_DEBUG_STARVE_TX, 0)
        mp.mp_debug_set(ctx, mp.MP_DEBUG_WAIT_BUDGET, 0)
        mp.mp_run_stages(ctx, mp.MP_STAGE_LIKELIHOOD)
        gn = mp.mp_get_buffer(ctx, mp.MP_BUF_GN)
        mp.mp_get_posterior(ctx)                  # error flag was cleared: no exception
    finally:
        mp.mp_destroy(ctx)
    P = room["P"]
    sn, sv, _, _ = oracle.point_normals(sc, P.r_cov, P.cov_k, P.cov_min)
    ref = oracle.likelihood(room["om"], room["w"].particles[:n], sc, sn, sv, P, amb_tol=1e-4)
    msg = check_sums(gn, ref)
    assert not msg, msg


def test_ragged_posterior_odd_sweeps(room, oracle):
    """The posterior stage (one cooperative launch, grid barriers between its
    sub-steps) on a ragged particle count with an odd number of sweeps,
    against the oracle's Eq. 11."""
    from paper_2404_16370_gb300 import mp
    n, K = 4099, 16
    rng = np.random.default_rng(31)
    ids = rng.integers(0, n, (n, K)).astype(np.int32)
    ids[rng.random((n, K)) < 0.3] = -1
    ids[:, 0] = np.arange(n)
    kk = rng.uniform(0.05, 1.0, (n, K)).astype(np.float32)
    kk[:, 0] = 1
    loglik = (-rng.uniform(0, 80, n)).astype(np.float32)
    logprior = -rng.uniform(0, 5, n)
    ctx = make_ctx(mp, room, n, post_iters=7)
    try:
        mp.mp_set_buffer(ctx, mp.MP_BUF_NBR_IDS, ids)
        mp.mp_set_buffer(ctx, mp.MP_BUF_NBR_K, kk)
        mp.mp_set_buffer(ctx, mp.MP_BUF_LOGLIK, loglik)
        mp.mp_set_buffer(ctx, mp.MP_BUF_LOG_PRIOR, logprior)
        mp.mp_run_stages(ctx, mp.MP_STAGE_POSTERIOR)
        post = mp.mp_get_buffer(ctx, mp.MP_BUF_POST)
        best, best_p = mp.mp_get_posterior(ctx)
    finally:
        mp.mp_destroy(ctx)
    _, p_ref, b_ref = oracle.posterior(logprior, loglik.astype(np.float64), ids, kk.astype(np.float64), 7,
                                       oracle.Params().post_floor)
    assert np.allclose(post, p_ref, rtol=1e-10, atol=1e-300)
    assert abs(post.sum() - 1) < 1e-12
    assert np.array_equal(best, room["w"].particles[b_ref]) and abs(best_p - p_ref[b_ref]) < 1e-12


def test_grid_barrier_gives_up_and_context_recovers(room):
    """A starved grid barrier (the posterior's first barrier waits for one CTA
    more than the grid): every CTA's bounded wait gives up after ~1 ms of SM
    clock, the kernel records the error and returns, and the host sees
    MP_ETIMEOUT; with the knob cleared the next step is normal."""
    from paper_2404_16370_gb300 import mp
    n = 4096
    sc = room["w"].scans[0]
    ctx = make_ctx(mp, room, n)
    try:
        mp.mp_debug_set(ctx, mp.MP_DEBUG_WAIT_BUDGET, 2_000_000)
        mp.mp_debug_set(ctx, mp.MP_DEBUG_STARVE_BARRIER, 1)
        mp.mp_step(ctx, sc)
        with pytest.raises(mp.MPError) as e:
            mp.mp_get_posterior(ctx)
        assert e.value.code == mp.MP_ETIMEOUT
        mp.mp_debug_set(ctx, mp.MP_DEBUG_STARVE_BARRIER, 0)
        mp.mp_debug_set(ctx, mp.MP_DEBUG_WAIT_BUDGET, 0)
        mp.mp_set_buffer(ctx, mp.MP_BUF_LOG_PRIOR, np.zeros(n))
        mp.mp_step(ctx, sc)
        best, best_p = mp.mp_get_posterior(ctx)   # error flag was cleared: no exception
        post = mp.mp_get_buffer(ctx, mp.MP_BUF_POST)
    finally:
        mp.mp_destroy(ctx)
    assert np.isfinite(post).all() and abs(post.sum() - 1) < 1e-12 and 0 < best_p <= 1
