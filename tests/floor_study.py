"""NRMSE floor of full-batch AP per reading of the data and of the regulariser, on the small
workload (256^2 object, 64^2 probe, 100 positions), with the FP64 oracle: flat start, true probe
held fixed, NRMSE to the ground truth every 10 iterations.  Regenerates the floor table of the
design notes:

    python tests/floor_study.py [iterations]      # ~2-3 min on 8 cores

Readings compared: the noiseless unclipped intensity itself ("ideal": what AP alone reaches),
the linear SLI comparator, and MNF with the default quantiser step (delta0 = 0.5) or none, for
the mean and weighted bases; each with alpha_O = alpha_P in {1e-3 (library default), 1e-4, 0}.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2608_01746_b300 import synth  # noqa: E402


def run(task):
    name, fused, sc, alpha, n_iter = task
    cfg = sc["cfg"]
    A = oracle.amplitudes(fused)
    obj = np.ones((cfg.M, cfg.M), complex)
    probe = sc["probe"].astype(complex)
    den = oracle.illumination(sc["probe"], sc["pos"], cfg.M)
    mask = den >= 0.1 * den.max()
    traj = []
    for it in range(n_iter):
        obj, probe, _ = oracle.iterate_once(obj, probe, sc["pos"], A, alpha, alpha, False)
        if (it + 1) % 10 == 0:
            traj.append(oracle.nrmse(obj, sc["obj"], mask))
    return name, alpha, traj


def main(n_iter: int = 800):
    import multiprocessing as mp
    sc = synth.make_scan("small")
    ideal = synth.make_scan("small", noise=False, clip=False)
    cfg = sc["cfg"]
    data = {"ideal": ideal["intensity"], "sli": oracle.sli_stack(sc["raw"], sc["times"], float(cfg.clip))}
    for bm in ("mean", "weighted"):
        for d0 in (0.5, 0.0):
            p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip), base_mode=bm, delta0=d0)
            data[f"mnf {bm} delta0={d0}"] = oracle.mnf_stack(sc["raw"], sc["times"], p)
    tasks = [(k, f, sc, a, n_iter) for k, f in data.items() for a in (1e-3, 1e-4, 0.0)]
    t0 = time.time()
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        res = pool.map(run, tasks)
    out = {}
    for name, alpha, traj in res:
        hit = next((10 * (i + 1) for i, v in enumerate(traj) if v <= 1e-2), None)
        out[f"{name} | alpha {alpha}"] = {"floor": round(min(traj), 5), "iterations_to_1e-2": hit,
                                          "every_100": [round(v, 4) for v in traj[9::10]]}
    print(json.dumps(out, indent=1))
    print(f"# {time.time() - t0:.0f} s", file=sys.stderr)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 800)
