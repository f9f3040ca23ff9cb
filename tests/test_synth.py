"""The shared input generator: shapes, seeding and photon scale."""
import numpy as np

from paper_2608_01746_b300 import synth


def test_small_workload_shapes_and_scale():
    sc = synth.make_scan("small")
    cfg = sc["cfg"]
    assert sc["raw"].shape == (100, 3, 64, 64) and sc["raw"].dtype == np.uint16
    assert sc["obj"].shape == (256, 256) and sc["probe"].shape == (64, 64)
    assert sc["pos"].min() >= 0 and sc["pos"].max() <= cfg.M - cfg.N
    assert sc["intensity"].max() == np.float64(cfg.peak)
    assert sc["raw"].max() == cfg.clip                    # the longest frame saturates
    amp = np.abs(sc["obj"])
    assert amp.min() >= 0.5 and amp.max() <= 1.0
    assert np.max(np.abs(np.angle(sc["obj"]))) <= np.pi / 2 + 1e-12


def test_seeded_and_deterministic():
    a = synth.make_scan("tiny")
    b = synth.make_scan("tiny")
    c = synth.make_scan("tiny", seed=5)
    assert np.array_equal(a["raw"], b["raw"])
    assert not np.array_equal(a["raw"], c["raw"])


def test_spiral_fits_object():
    pos = synth.spiral_positions(1024, 256, 1600)
    assert pos.shape == (1600, 2)
    assert pos.min() >= 0 and pos.max() <= 768
    d = np.hypot(*(pos[1:] - pos[:1]).T)
    assert d.max() <= 384 * np.sqrt(2) + 1


def test_batched_configs_follow_the_workload_recipe():
    """64 datasets, probe sides from {64, 128, 256}, n x n rasters with 7 <= n <= 30 (49-900
    positions), object sides 256-1024 that hold every patch, same draw for the same seed."""
    from paper_2608_01746_b300 import synth
    cfgs = synth.batched_configs()
    assert len(cfgs) == 64
    assert {c.N for c in cfgs} == {64, 128, 256}
    for c in cfgs:
        assert 7 <= c.n_side <= 30 and 49 <= c.n_pos <= 900
        assert 256 <= c.M <= 1024 and c.M % 32 == 0
        assert c.step == c.N // 8 and c.radius == 5.0 * c.N / 16.0
        assert c.N + (c.n_side - 1) * c.step + 2 * c.jitter <= c.M
    again = synth.batched_configs()
    assert [(c.N, c.n_side, c.M) for c in cfgs] == [(c.N, c.n_side, c.M) for c in again]
    other = synth.batched_configs(seed=7)
    assert [(c.N, c.n_side) for c in cfgs] != [(c.N, c.n_side) for c in other]
