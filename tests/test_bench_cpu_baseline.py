"""The CPU-baseline machinery of bench.py (no GPU): the oracle's per-position steps spread over
a spawn process pool give exactly what the oracle computes in one process."""
import numpy as np

import oracle
from paper_2608_01746_b300 import synth


def test_pooled_iteration_and_fusion_match_the_oracle():
    import bench
    sc = synth.make_scan("tiny")
    cfg = sc["cfg"]
    p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip))
    fused = oracle.mnf_stack(sc["raw"], sc["times"], p)
    A = oracle.amplitudes(fused)
    obj = np.ones((cfg.M, cfg.M), complex)
    probe = sc["probe"].astype(complex)
    ro, rp, re = oracle.iterate_once(obj, probe, sc["pos"], A, 1e-3, 1e-3, True)
    pool = bench.OraclePool(A, 2)
    try:
        po, pp, pe = pool.iteration(obj, probe, sc["pos"])
        pf = pool.fuse(sc["raw"], sc["times"], p)
    finally:
        pool.close()
    assert np.array_equal(po, ro) and np.array_equal(pp, rp)
    assert pe == np.float64(re) or abs(pe - re) <= 1e-12 * abs(re)      # chunk sums: summation order
    assert np.array_equal(np.stack(pf), fused)
