"""Batches of uneven datasets (ptycho_batch_*) against the same datasets iterated one handle at a
time.  A batch runs the same per-position arithmetic (the multi-dataset exit-wave launch processes
each position exactly as the single-dataset launch does), so objects and probes must agree bit for
bit, with and without graph capture and autotuning; the single-handle paths are themselves
checked against the FP64 oracle in the other GPU tests."""
import dataclasses

import numpy as np
import pytest

from paper_2608_01746_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_01746_b300 import api as a
    a.lib()
    return a


# (config, fft path, probe_update_start): N = 16 / 64 / 128 radix classes, the N = 64
# tensor-core class, an N = 256 dataset on its own TMA launch, a mixed-state dataset (8 modes)
DATASETS = [("tiny", "radix_fp32", 0), ("small", "radix_fp32", 3), ("mid", "radix_fp32", 0),
            ("small", "dftgemm_bf16x3", 0), ("mid", "dftgemm_bf16x3", 3), ("lab40", "radix_fp32", 0),
            ("mixed_small", "radix_fp32", 0), ("mid128", "radix_fp32", 3)]


def _scan(name, seed):
    if name == "lab40":
        cfg = dataclasses.replace(synth.CONFIGS["lab"], J=40)
        sc = synth.make_scan_torch(cfg, seed=seed)
        return cfg, sc, sc["raw"]
    cfg = synth.CONFIGS[name]
    sc = synth.make_scan(cfg, seed=seed)
    return cfg, sc, torch.from_numpy(sc["raw"].astype(np.uint16)).cuda()


@pytest.fixture(scope="module")
def inputs(api):
    out = []
    for i, (name, fft, pus) in enumerate(DATASETS):
        cfg, sc, raw = _scan(name, 500 + i)
        fused = api.fuse_stack(raw, cfg.times, api.fuse_params(levels=cfg.levels, clip=float(cfg.clip)))
        rng = np.random.default_rng(i)
        M = cfg.M
        obj0 = (1 + 0.1 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))).astype(np.complex64)
        out.append(dict(fused=fused, pos=sc["pos"], obj0=obj0, probe0=sc["probe"].astype(np.complex64),
                        fft=fft, pus=pus))
    torch.cuda.synchronize()
    return out


def _handles(api, inputs):
    return [api.ptycho_init(d["fused"], d["pos"], d["obj0"], d["probe0"], probe_update_start=d["pus"],
                            fft_path=d["fft"]) for d in inputs]


@pytest.fixture(scope="module")
def reference(api, inputs):
    """Each dataset iterated alone: 2 + 4 iterations (the probe switches on at iteration 3 for
    some datasets, so a captured graph must be re-captured)."""
    hs = _handles(api, inputs)
    errs = []
    for h in hs:
        api.ptycho_iterate(h, 2)
        errs.append(api.ptycho_iterate(h, 4)[-1])
    res = [(api.ptycho_get_object(h), api.ptycho_get_probe(h)) for h in hs]
    for h in hs:
        api.ptycho_destroy(h)
    return res, np.array(errs)


@pytest.mark.parametrize("graph,autotune", [(False, False), (True, False), (True, True)])
def test_batch_matches_individual_handles(api, inputs, reference, graph, autotune):
    ref, ref_err = reference
    hs = _handles(api, inputs)
    b = api.ptycho_batch_create(hs, graph=graph, autotune=autotune)
    if autotune:
        desc = api.ptycho_batch_describe(b)
        print("autotune:", desc)
        assert "class_radix64_grid" in desc and "tma_rows_n256" in desc
    api.ptycho_batch_iterate(b, 2)
    err = api.ptycho_batch_iterate(b, 4)
    for i, h in enumerate(hs):
        o, p = api.ptycho_get_object(h), api.ptycho_get_probe(h)
        assert np.array_equal(o, ref[i][0]), DATASETS[i]
        assert np.array_equal(p, ref[i][1]), DATASETS[i]
    # the N = 256 kernel accumulates each thread's error terms in FP32; the autotuned rows per
    # TMA stage change which terms a thread sums, so that error agrees to FP32 accumulation order
    np.testing.assert_allclose(err, ref_err, rtol=1e-6 if autotune else 0)
    # a handle stays usable on its own after the batch
    e1 = api.ptycho_iterate(hs[0], 1)
    assert np.isfinite(e1).all()
    api.ptycho_batch_destroy(b)
    for h in hs:
        api.ptycho_destroy(h)


def test_batch_rejects_epie_and_duplicates(api, inputs):
    d = inputs[0]
    h = api.ptycho_init(d["fused"], d["pos"], d["obj0"], d["probe0"], algorithm="epie_colour")
    h2 = api.ptycho_init(d["fused"], d["pos"], d["obj0"], d["probe0"])
    with pytest.raises(api.PtychoError):
        api.ptycho_batch_create([h2, h])
    with pytest.raises(api.PtychoError):
        api.ptycho_batch_create([h2, h2])
    api.ptycho_destroy(h)
    api.ptycho_destroy(h2)
