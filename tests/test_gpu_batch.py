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


@pytest.mark.parametrize("graph,autotune,one", [(False, False, False), (True, False, False), (True, True, False),
                                                (False, False, True), (True, True, True)])
def test_batch_matches_individual_handles(api, inputs, reference, graph, autotune, one):
    """one: every single-mode radix dataset's exit waves in one persistent launch (all N)."""
    ref, ref_err = reference
    hs = _handles(api, inputs)
    b = api.ptycho_batch_create(hs, graph=graph, autotune=autotune, one_launch=one)
    if autotune and not one:
        desc = api.ptycho_batch_describe(b)
        print("autotune:", desc)
        assert "class_radix64_grid" in desc and "tma_rows_n256" in desc
        assert '"one_launch"' in desc              # the per-size launches against the one launch
    api.ptycho_batch_iterate(b, 2)
    err = api.ptycho_batch_iterate(b, 4)
    for i, h in enumerate(hs):
        o, p = api.ptycho_get_object(h), api.ptycho_get_probe(h)
        assert np.array_equal(o, ref[i][0]), DATASETS[i]
        assert np.array_equal(p, ref[i][1]), DATASETS[i]
    # each thread accumulates its error terms in FP32; the autotuned rows per TMA stage (N = 256)
    # and the one launch's 128-thread quarters (N <= 64) change which terms a thread sums, so the
    # error then agrees to FP32 accumulation order
    np.testing.assert_allclose(err, ref_err, rtol=1e-6 if (autotune or one) else 0)
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


def test_batch_graph_survives_handle_iterations(api, inputs):
    """A captured batch iteration keeps working after the handles are iterated on their own in
    between (ptycho_iterate with more iterations than before grows its own error buffer; the
    graph must not depend on it): batch 2, alone 4, batch 3 == alone 2 + 4 + 3."""
    ref_h = _handles(api, inputs)
    for h in ref_h:
        api.ptycho_iterate(h, 2)
        api.ptycho_iterate(h, 4)
    ref_err = np.array([api.ptycho_iterate(h, 3)[-1] for h in ref_h])
    ref = [(api.ptycho_get_object(h), api.ptycho_get_probe(h)) for h in ref_h]
    for h in ref_h:
        api.ptycho_destroy(h)
    hs = _handles(api, inputs)
    b = api.ptycho_batch_create(hs, graph=True)
    api.ptycho_batch_iterate(b, 2)
    for h in hs:
        api.ptycho_iterate(h, 4)
    err = api.ptycho_batch_iterate(b, 3)
    for i, h in enumerate(hs):
        assert np.array_equal(api.ptycho_get_object(h), ref[i][0]), DATASETS[i]
        assert np.array_equal(api.ptycho_get_probe(h), ref[i][1]), DATASETS[i]
    np.testing.assert_array_equal(err, ref_err)
    api.ptycho_batch_destroy(b)
    for h in hs:
        api.ptycho_destroy(h)


# One dataset of every exit-wave class, fused by the oracle: (config, fft path, probe_update_start,
# tolerance on object and probe after 2 + 3 iterations).  The split-BF16 form is held to its own
# bound, 12 x 2^-16 per iteration (see test_gpu_dftgemm.py).
ORACLE_DATASETS = [("tiny", "radix_fp32", 0, 1e-5), ("small", "radix_fp32", 3, 1e-5),
                   ("small", "dftgemm_bf16x3", 0, 5 * 12 * 2.0 ** -16), ("mid128", "radix_fp32", 3, 1e-5),
                   ("mid128", "dftgemm_bf16x3", 0, 5 * 12 * 2.0 ** -16), ("lab12", "radix_fp32", 0, 1e-5)]


def test_batch_classes_match_the_oracle(api):
    """Every class of a graph-captured, autotuned batch (N = 16, 64 and 128 radix launches, the
    N = 64 and 128 tensor-core forms, an N = 256 dataset on its own TMA launch) against the FP64
    oracle directly, on fusion computed by the oracle."""
    import oracle
    from tests.parity_helpers import rel_l2
    data = []
    for i, (name, fft, pus, tol) in enumerate(ORACLE_DATASETS):
        if name == "lab12":
            cfg = dataclasses.replace(synth.CONFIGS["lab"], J=12)
            sc = synth.make_scan_torch(cfg, seed=900 + i, device="cpu")
            raw = sc["raw"].numpy()
        else:
            cfg = synth.CONFIGS[name]
            sc = synth.make_scan(cfg, seed=900 + i)
            raw = sc["raw"]
        p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip))
        fused = oracle.mnf_stack(raw, cfg.times, p).astype(np.float32)
        rng = np.random.default_rng(100 + i)
        M = cfg.M
        obj0 = (1 + 0.1 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))).astype(np.complex64)
        data.append(dict(fused=fused, pos=sc["pos"], obj0=obj0, probe0=sc["probe"].astype(np.complex64),
                         fft=fft, pus=pus, tol=tol))
    hs = [api.ptycho_init(torch.from_numpy(d["fused"]).cuda(), d["pos"], d["obj0"], d["probe0"],
                          probe_update_start=d["pus"], fft_path=d["fft"]) for d in data]
    b = api.ptycho_batch_create(hs, graph=True, autotune=True)
    api.ptycho_batch_iterate(b, 2)
    api.ptycho_batch_iterate(b, 3)
    for d, h, spec in zip(data, hs, ORACLE_DATASETS):
        ro, rp, _ = oracle.reconstruct(d["fused"].astype(np.float64), d["pos"], d["obj0"].astype(np.complex128),
                                       d["probe0"].astype(np.complex128), 5, 1e-3, 1e-3, d["pus"])
        eo = rel_l2(api.ptycho_get_object(h), ro)
        ep = rel_l2(api.ptycho_get_probe(h), rp)
        print(spec, f"object {eo:.2e} probe {ep:.2e}")
        assert eo <= d["tol"] and ep <= d["tol"], (spec, eo, ep)
    api.ptycho_batch_destroy(b)
    for h in hs:
        api.ptycho_destroy(h)
