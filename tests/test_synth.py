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
