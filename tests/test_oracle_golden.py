"""The oracle's defaults against the constants the paper prints
(tests/golden/paper_constants.json, each entry with its citation)."""
import json
import os

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_printed_constants(oracle):
    P = oracle.Params()
    assert P.sigma_r == G["sigma_r_per_rad"]["value"]
    assert P.sigma_t == G["sigma_t_per_m"]["value"]
    assert P.post_iters == G["posterior_iterations"]["value"]
    assert oracle.Params.box_room().res == G["nnf_resolution_indoor_m"]["value"]
    assert oracle.Params.outdoor().res == G["nnf_resolution_outdoor_m"]["value"]
    # 2^20 particles hash into 2^20 buckets in the paper-scale preset
    assert 1 << oracle.Params.outdoor(G["particles"]["value"]).nb_log2 == G["particles"]["value"]


def test_oracle_filter_runs_and_normalises(oracle):
    import numpy as np
    from paper_2404_16370_gb300 import synth
    w = synth.box_room_workload(n_particles=256, n_steps=2)
    P = oracle.Params.box_room(256)
    f = oracle.OracleFilter(oracle.OracleMap(w.map_points, P), P, w.particles.copy())
    for s in range(2):
        out = f.step(w.scans[s], w.odom[s], w.odom_cov[s])
        assert abs(out["post"].sum() - 1) < 1e-12
        assert np.all(out["nbr_ids"][:, 0] == np.arange(256))
    out = f.step(np.zeros((0, 3), np.float32))      # blackout step: prediction + smoothing only
    assert abs(out["post"].sum() - 1) < 1e-12
