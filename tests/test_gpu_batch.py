"""Batched instances (mp_batch_*) and the likelihood's scan split: the split
sums equal the unsplit ones up to summation order; a batch step equals the
same step taken instance by instance with mp_step (bit for bit with split 1);
the autotuned batch runs with valid splits and posteriors; a starved grid
barrier in the batched posterior is reported for every instance; contexts
sharing one device map (mp_init_map_shared) compute what contexts with their
own copies compute, outlive the context that built the map, and refuse map
parameters that differ; an instance with the preconditioned SVGD reading
batches bit for bit too."""
import numpy as np
import pytest

from paper_2404_16370_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _room_instance(seed, n_part, n_rays):
    room = synth.box_room(seed)
    gt = synth.box_room_gt_pose(room, seed + 100)
    sc = synth.scan(room, gt, synth.spherical_dirs(n_rays), 0.02, seed + 200)
    parts = synth.box_room_particles(n_part, seed + 300, room.half)
    return room, sc, parts


def test_likelihood_split_matches_unsplit():
    from paper_2404_16370_gb300 import mp
    room, sc, parts = _room_instance(1, 4096, 2048)
    ctx = mp.mp_init_map(room.map_points, mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, 4096))
    try:
        mp.mp_init_particles(ctx, 4096, poses=parts)
        mp.mp_set_scan(ctx, sc)
        mp.mp_run_stages(ctx, mp.MP_STAGE_SCAN | mp.MP_STAGE_LSH | mp.MP_STAGE_SORT)
        out = {}
        for split in (1, 3, 8):
            mp.mp_set_likelihood_split(ctx, split)
            mp.mp_run_stages(ctx, mp.MP_STAGE_LIKELIHOOD)
            out[split] = mp.mp_get_buffer(ctx, mp.MP_BUF_GN).astype(np.float64)
    finally:
        mp.mp_destroy(ctx)
    ref = out[1]
    scale = np.abs(ref).max(axis=0, keepdims=True) + 1e-6
    for split in (3, 8):
        assert np.array_equal(out[split][:, 28], ref[:, 28])      # inlier counts: exact
        assert np.all(np.abs(out[split] - ref) <= 2e-5 * scale)


def _instances(stream, specs):
    """Box-room instances; every context on `stream` (instances never run
    concurrently: the batch and the eager steps are ordered on one stream)."""
    from paper_2404_16370_gb300 import mp
    ctxs, data = [], []
    for seed, n_part, n_rays in specs:
        room, sc, parts = _room_instance(seed, n_part, n_rays)
        ctx = mp.mp_init_map(room.map_points, mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, n_part),
                             cuda_stream=stream)
        mp.mp_init_particles(ctx, n_part, poses=parts)
        ctxs.append(ctx)
        data.append((sc, parts))
    return ctxs, data


SPECS = [(1, 1024, 512), (2, 3000, 700), (3, 4096, 512)]


def _odometry(n, step):
    rng = np.random.default_rng(1000 + step)
    T = np.tile(np.eye(4), (n, 1, 1))
    T[:, :3, 3] = rng.normal(0, 0.02, (n, 3))
    cov = np.tile(np.diag([1e-6] * 3 + [1e-4] * 3), (n, 1, 1))
    return T, cov


def _compare(A, B):
    from paper_2404_16370_gb300 import mp
    for i in range(len(A)):
        pa, prob_a = mp.mp_get_posterior(A[i])
        pb, prob_b = mp.mp_get_posterior(B[i])
        for which in (mp.MP_BUF_POSES, mp.MP_BUF_POST, mp.MP_BUF_NBR_IDS, mp.MP_BUF_GN):
            assert np.array_equal(mp.mp_get_buffer(A[i], which), mp.mp_get_buffer(B[i], which)), (i, which)
        assert np.array_equal(pa, pb) and prob_a == prob_b


def test_batch_step_equals_sequential_steps(torch):
    """Three instances stepped by the grouped batch graph equal the same
    instances stepped one by one with mp_step, bit for bit."""
    from paper_2404_16370_gb300 import mp
    st = mp.mp_stream_create()
    A, data = _instances(st, SPECS)
    B, _ = _instances(st, SPECS)
    batch = mp.mp_batch_create(A, [len(d[0]) for d in data], st)
    try:
        for step in range(3):
            T, cov = _odometry(len(SPECS), step)
            mp.mp_batch_step(batch, [d[0] for d in data], T, cov)
            for i, ctx in enumerate(B):
                mp.mp_step(ctx, data[i][0], T[i], cov[i])
        for i in range(len(SPECS)):
            assert mp.mp_batch_split(batch, i) == 1
        _compare(A, B)
    finally:
        mp.mp_batch_destroy(batch)
        for c in A + B:
            mp.mp_destroy(c)
        mp.mp_stream_destroy(st)


def test_batch_mixed_presets_equal_sequential_steps(torch):
    """Instances of different presets and list lengths (a box room with
    K = 16 and an outdoor scene with K = 32, one with an odd number of
    posterior sweeps) in one batch: bit for bit the eager steps."""
    from paper_2404_16370_gb300 import mp
    st = mp.mp_stream_create()
    sc_out = synth.outdoor(21, n_map=60_000)
    gt = synth.outdoor_trajectory(1, 0, seed=22, scene=sc_out)[0]
    scan_out = synth.scan(sc_out, gt, synth.lidar_dirs(16, 128), 0.03, 23, dropout=0.1, max_range=60.0).astype(np.float32)
    parts_out = synth.outdoor_particles(sc_out, 2500, 24)
    room, scan_room, parts_room = _room_instance(5, 2048, 600)

    def make():
        p_room = mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, 2048)
        p_room.post_iters = 7
        c1 = mp.mp_init_map(room.map_points, p_room, cuda_stream=st)
        mp.mp_init_particles(c1, 2048, poses=parts_room)
        c2 = mp.mp_init_map(sc_out.map_points, mp.mp_default_params(mp.MP_PRESET_OUTDOOR, 2500), cuda_stream=st)
        mp.mp_init_particles(c2, 2500, poses=parts_out)
        return [c1, c2]

    A, B = make(), make()
    scans = [scan_room, scan_out]
    batch = mp.mp_batch_create(A, [len(s) for s in scans], st)
    try:
        for step in range(3):
            T, cov = _odometry(2, step)
            mp.mp_batch_step(batch, scans, T, cov)
            for i, ctx in enumerate(B):
                mp.mp_step(ctx, scans[i], T[i], cov[i])
        _compare(A, B)
    finally:
        mp.mp_batch_destroy(batch)
        for c in A + B:
            mp.mp_destroy(c)
        mp.mp_stream_destroy(st)


def test_autotuned_batch_runs(torch):
    from paper_2404_16370_gb300 import mp
    specs = [(4, 2048, 4096), (5, 8192, 2048), (6, 1024, 512)]
    st = mp.mp_stream_create()
    A, data = _instances(st, specs)
    batch = mp.mp_batch_create(A, [len(d[0]) for d in data], st, tune_scans=[d[0] for d in data])
    try:
        splits = [mp.mp_batch_split(batch, i) for i in range(len(specs))]
        assert all(s in (1, 2, 4, 8, 16) for s in splits)
        for step in range(4):
            mp.mp_batch_step(batch, [d[0] for d in data])
        for i, ctx in enumerate(A):
            post = mp.mp_get_buffer(ctx, mp.MP_BUF_POST)
            assert np.isfinite(post).all() and abs(post.sum() - 1) < 1e-9
        print("\nsplits", splits)
    finally:
        mp.mp_batch_destroy(batch)
        for c in A:
            mp.mp_destroy(c)
        mp.mp_stream_destroy(st)


def test_batch_refuses_outside_steps(torch):
    """A batched context stepped with mp_step is refused by the next batch
    step (its neighbour-list index no longer matches the captured graph)."""
    from paper_2404_16370_gb300 import mp
    st = mp.mp_stream_create()
    A, data = _instances(st, SPECS[:2])
    batch = mp.mp_batch_create(A, [len(d[0]) for d in data], st)
    try:
        mp.mp_batch_step(batch, [d[0] for d in data])
        mp.mp_step(A[0], data[0][0])
        with pytest.raises(mp.MPError):
            mp.mp_batch_step(batch, [d[0] for d in data])
    finally:
        mp.mp_batch_destroy(batch)
        for c in A:
            mp.mp_destroy(c)
        mp.mp_stream_destroy(st)


def test_batch_grid_barrier_timeout_reported_for_every_instance(torch):
    """The batched posterior is one cooperative launch over all instances.
    With the first instance's barrier knob set when the batch is created, its
    first grid barrier waits for one CTA more than the grid: every CTA gives
    up, and every instance reports MP_ETIMEOUT."""
    from paper_2404_16370_gb300 import mp
    st = mp.mp_stream_create()
    A, data = _instances(st, SPECS)
    mp.mp_debug_set(A[0], mp.MP_DEBUG_WAIT_BUDGET, 2_000_000)
    mp.mp_debug_set(A[0], mp.MP_DEBUG_STARVE_BARRIER, 1)
    batch = mp.mp_batch_create(A, [len(d[0]) for d in data], st)
    try:
        mp.mp_batch_step(batch, [d[0] for d in data])
        for ctx in A:
            with pytest.raises(mp.MPError) as e:
                mp.mp_get_posterior(ctx)
            assert e.value.code == mp.MP_ETIMEOUT
    finally:
        mp.mp_batch_destroy(batch)
        for c in A:
            mp.mp_destroy(c)
        mp.mp_stream_destroy(st)


def _room_params(n, **over):
    from paper_2404_16370_gb300 import mp
    return mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, n, **over)


def test_shared_map_equals_own_map_and_outlives_its_source():
    """Two contexts on one device map (the second made by mp_init_map_shared,
    with other K and particle count) against two contexts with their own
    copies: bit for bit after 3 steps, with the map's source destroyed before
    the shared context steps."""
    from paper_2404_16370_gb300 import mp
    room, sc, parts = _room_instance(7, 3000, 700)
    p1, p2 = _room_params(3000), _room_params(2048, K=8, C=8)
    src = mp.mp_init_map(room.map_points, p1)
    shared = mp.mp_init_map_shared(src, p2)
    own = mp.mp_init_map(room.map_points, p2)
    try:
        assert np.array_equal(mp.mp_get_buffer(shared, mp.MP_BUF_MAP_NORMALS),
                              mp.mp_get_buffer(own, mp.MP_BUF_MAP_NORMALS))
        mp.mp_destroy(src)
        src = None
        for c in (shared, own):
            mp.mp_init_particles(c, 2048, poses=parts[:2048])
        for step in range(3):
            T, cov = _odometry(1, step)
            for c in (shared, own):
                mp.mp_step(c, sc, T[0], cov[0])
        _compare([shared], [own])
    finally:
        for c in (src, shared, own):
            if c is not None:
                mp.mp_destroy(c)


def test_shared_map_refuses_other_map_parameters():
    from paper_2404_16370_gb300 import mp
    room, _, _ = _room_instance(8, 512, 256)
    src = mp.mp_init_map(room.map_points, _room_params(512))
    try:
        for over in ({"nnf_res": 0.2}, {"r_max": 0.5}, {"r_cov": 0.5}, {"cov_k": 8}):
            with pytest.raises(mp.MPError) as e:
                mp.mp_init_map_shared(src, _room_params(512, **over))
            assert e.value.code == mp.MP_EINVAL
    finally:
        mp.mp_destroy(src)


def test_batch_on_shared_maps_equals_sequential_steps(torch):
    """A batch whose instances share device maps (two per map) equals the same
    instances with their own maps stepped one by one, bit for bit."""
    from paper_2404_16370_gb300 import mp
    st = mp.mp_stream_create()
    specs = [(1, 1024, 512), (1, 2000, 600), (2, 1500, 512), (2, 4096, 700)]
    data = [_room_instance(*sp) for sp in specs]
    A, B = [], []
    try:
        for k, (room, sc, parts) in enumerate(data):
            n = specs[k][1]
            if k % 2 == 0:
                A.append(mp.mp_init_map(room.map_points, _room_params(n), cuda_stream=st))
            else:
                A.append(mp.mp_init_map_shared(A[k - 1], _room_params(n), cuda_stream=st))
            B.append(mp.mp_init_map(room.map_points, _room_params(n), cuda_stream=st))
            for c in (A[k], B[k]):
                mp.mp_init_particles(c, n, poses=parts)
        scans = [d[1] for d in data]
        batch = mp.mp_batch_create(A, [len(s) for s in scans], st)
        try:
            for step in range(3):
                T, cov = _odometry(len(specs), step)
                mp.mp_batch_step(batch, scans, T, cov)
                for i, c in enumerate(B):
                    mp.mp_step(c, scans[i], T[i], cov[i])
            _compare(A, B)
        finally:
            mp.mp_batch_destroy(batch)
    finally:
        for c in A + B:
            mp.mp_destroy(c)
        mp.mp_stream_destroy(st)


def test_batch_with_preconditioned_svgd_equals_sequential_steps(torch):
    """One instance with the preconditioned SVGD reading (svgd_precond = 1:
    the solve stores each particle's inverse, SVGD multiplies the repulsion
    by it) batched with one without: bit for bit the eager steps."""
    from paper_2404_16370_gb300 import mp
    st = mp.mp_stream_create()
    specs = [(9, 2048, 600), (10, 3000, 512)]
    data = [_room_instance(*sp) for sp in specs]

    def make():
        cs = []
        for k, (room, sc, parts) in enumerate(data):
            n = specs[k][1]
            cs.append(mp.mp_init_map(room.map_points, _room_params(n, svgd_precond=1 - k), cuda_stream=st))
            mp.mp_init_particles(cs[-1], n, poses=parts)
        return cs

    A, B = make(), make()
    scans = [d[1] for d in data]
    try:
        batch = mp.mp_batch_create(A, [len(s) for s in scans], st)
        try:
            for step in range(3):
                T, cov = _odometry(len(specs), step)
                mp.mp_batch_step(batch, scans, T, cov)
                for i, c in enumerate(B):
                    mp.mp_step(c, scans[i], T[i], cov[i])
            _compare(A, B)
        finally:
            mp.mp_batch_destroy(batch)
    finally:
        for c in A + B:
            mp.mp_destroy(c)
        mp.mp_stream_destroy(st)
