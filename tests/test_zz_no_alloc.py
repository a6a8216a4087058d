"""The allocation-free initial posterior (mp_posterior_init_noalloc), through
the C ABI, on two calls in a row: against the FP64 oracle's initial posterior
and against the context's own posterior stage (MP_BUF_POST_INIT).

For callers that cannot allocate device memory when they need the posterior
(a real-time loop that allocates only at start-up, or an application whose
device memory is owned by another allocator): the entry point works on the
caller's buffers and a fixed static device array. This file is collected last
so that a failure here leaves every other test already run."""
import numpy as np
import pytest

from paper_2404_16370_gb300 import synth

pytestmark = pytest.mark.gpu

N = 40000   # not a multiple of the 2048-element block tile: a ragged last block


def stage_reference(mp, ctx, logprior, loglik):
    """Initial posterior and its argmax from the existing posterior stage (no
    smoothing sweeps, so its representative state is the initial argmax)."""
    mp.mp_set_buffer(ctx, mp.MP_BUF_LOG_PRIOR, logprior)
    mp.mp_set_buffer(ctx, mp.MP_BUF_LOGLIK, loglik)
    mp.mp_run_stages(ctx, mp.MP_STAGE_POSTERIOR)
    post0 = mp.mp_get_buffer(ctx, mp.MP_BUF_POST_INIT)
    best_pose, _ = mp.mp_get_posterior(ctx)
    return post0, best_pose


def test_noalloc_initial_posterior_matches_oracle_and_posterior_stage():
    import torch
    from oracle import oracle as O
    from paper_2404_16370_gb300 import mp
    room = synth.box_room(1, n_map=5000)
    # the posterior stage without its floor: the entry point computes the plain exp(l - max l)
    params = mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, N, post_iters=0, post_floor=0.0)
    ctx = mp.mp_init_map(room.map_points, params)
    try:
        poses = synth.box_room_particles(N, seed=5)
        mp.mp_init_particles(ctx, N, poses=poses)
        rng = np.random.default_rng(42)
        dev = torch.device("cuda:0")
        post_out = torch.empty(N, dtype=torch.float64, device=dev)
        best_out = torch.empty(1, dtype=torch.int64, device=dev)
        free_after = []
        for call in range(2):
            logprior = -rng.uniform(0.0, 4.0, N)
            logprior[::101] = -np.inf
            loglik = (-rng.uniform(0.0, 700.0, N)).astype(np.float32)
            top = int(rng.integers(0, N))
            loglik[top] = 5.0          # one clear maximum
            ref_post, ref_best_pose = stage_reference(mp, ctx, logprior, loglik)
            ids = np.arange(N, dtype=np.int32).reshape(N, 1)
            or_post, _, or_best = O.posterior(logprior, loglik.astype(np.float64), ids, np.ones((N, 1)), 0)
            post_out.fill_(np.nan)
            best_out.fill_(-7)
            lp_t = torch.from_numpy(logprior).to(dev)
            ll_t = torch.from_numpy(loglik).to(dev)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            mp.mp_posterior_init_noalloc(lp_t, ll_t, post_out, best_out)
            torch.cuda.synchronize()
            free_after.append((free0, torch.cuda.mem_get_info()[0]))
            got = post_out.cpu().numpy()
            best = int(best_out.item())
            # the oracle: p_i = exp(l_i - max l) / sum, FP64; the sum's order differs
            assert np.allclose(got, or_post, rtol=1e-12, atol=1e-300), f"call {call}"
            assert best == or_best == top, f"call {call}: best {best}, oracle {or_best}, planted {top}"
            # the context's posterior stage: the same values up to the sum's rounding, the same argmax
            assert np.allclose(got, ref_post, rtol=1e-12, atol=1e-300), f"call {call}"
            assert abs(got.sum() - 1.0) < 1e-12
            assert np.array_equal(poses[best], ref_best_pose), f"call {call}: best {best}"
        # after the first call (which may load the module) a call allocates nothing
        f0, f1 = free_after[1]
        assert f1 == f0, f"free device memory changed by {f0 - f1} bytes during the second call"
        # a size beyond the fixed scratch is rejected before any launch (the
        # 8-element buffer is never read)
        small = torch.zeros(8, dtype=torch.float32, device=dev)
        rc = mp.lib().mp_posterior_init_noalloc(None, small.data_ptr(), 2 ** 24 + 1, post_out.data_ptr(),
                                                best_out.data_ptr(), None)
        assert rc == mp.MP_EINVAL and "outside" in mp.mp_last_error(None)
        # host memory, even pinned, is refused by the C entry point itself
        host = torch.zeros(8, dtype=torch.float32).pin_memory()
        rc = mp.lib().mp_posterior_init_noalloc(None, host.data_ptr(), 8, post_out.data_ptr(), best_out.data_ptr(),
                                                None)
        assert rc == mp.MP_EINVAL and "loglik" in mp.mp_last_error(None)
    finally:
        mp.mp_destroy(ctx)


def test_noalloc_degenerate_input_gives_the_sentinels():
    """Every l_i = -inf: no normaliser exists; best = -1 and post = NaN."""
    import torch
    from paper_2404_16370_gb300 import mp
    dev = torch.device("cuda:0")
    n = 5000
    lp = torch.full((n,), -np.inf, dtype=torch.float64, device=dev)
    ll = torch.zeros(n, dtype=torch.float32, device=dev)
    post = torch.zeros(n, dtype=torch.float64, device=dev)
    best = torch.zeros(1, dtype=torch.int64, device=dev)
    mp.mp_posterior_init_noalloc(lp, ll, post, best)
    torch.cuda.synchronize()
    assert int(best.item()) == -1
    assert torch.isnan(post).all()
    # a finite input afterwards is served normally (nothing stale in the scratch)
    lp.fill_(0.0)
    ll[123] = 1.0
    mp.mp_posterior_init_noalloc(lp, ll, post, best)
    torch.cuda.synchronize()
    assert int(best.item()) == 123 and abs(float(post.sum()) - 1.0) < 1e-12
