"""Batched persistent march: bit-identity with single-grid runs, CUDA-graph
replay, parity with the oracle, bounded waits and the autotuner."""
import numpy as np
import pytest
import torch

import oracle
from paper_2306_15678_gb300 import beams, capi, configs
from paper_2306_15678_gb300.batch import Batch
from paper_2306_15678_gb300.grid import Grid

pytestmark = pytest.mark.gpu


def mixed_beams(sizes=(256, 512, 1024, 2048, 512, 4096), seed=11):
    rng = np.random.default_rng(seed)
    out = []
    for b, n in enumerate(sizes):
        w0 = float(rng.uniform(0.3, 0.8))
        cfg = configs.physics(n, 8 * w0, 0.5, configs.ALL_TERMS)
        cfg["beam"] = dict(w0=w0, P=float(rng.uniform(20, 200)) * configs.critical_power(), amp=0.05,
                           ell_cells=0.05 / (8 * w0 / n), seed=900 + b, phase=0.1, phase_seed=950 + b)
        out.append(cfg)
    return out


def single(cfg, U, nsteps, radix=16):
    with Grid(cfg, precision="fp32") as g:
        if radix == 8:
            capi.nlse_set_row_radix(g.h, 8)
            capi.nlse_set_column_tile(g.h, capi.NLSE_COL_R8 | 1)
        return g.load(U).step(nsteps).field()


@pytest.mark.parametrize("threads,radix,per_thread", [(256, 16, 0), (512, 16, 0), (256, 8, 0), (512, 8, 0),
                                                      (128, 16, 0), (256, 16, 1), (512, 8, 1)])
def test_batched_beams_bit_identical_to_single_grids(threads, radix, per_thread):
    """Every launch shape (threads, radix) and both column paths (staged by
    bulk tensor copies for n >= 512, or per-thread) give each beam the bits of
    the same beam on its own grid with the same radix."""
    sizes = ((256, 512, 1024, 2048, 512, 4096) if threads == 512 or (threads == 256 and radix == 16)
             else (256, 512, 1024, 2048, 512))
    cfgs = mixed_beams(sizes)
    fields = [beams.make_field(c).astype(np.complex64) for c in cfgs]
    with Batch(cfgs, {"threads": threads, "radix": radix, "per_thread_columns": per_thread}) as b:
        for i, U in enumerate(fields):
            b.load(i, U)
        b.step(7).step(5)
        assert b.status() == capi.NLSE_OK
        assert b.steps_taken == 12
        for i, (c, U) in enumerate(zip(cfgs, fields)):
            assert np.array_equal(b.field(i), single(c, U, 12, radix)), i
            assert np.array_equal(b.field(i, device=True).cpu().numpy(), b.field(i))


def test_shapes_too_narrow_for_a_size_are_refused():
    cfgs = mixed_beams((4096,))
    for tuning in ({"threads": 256, "radix": 8}, {"threads": 128, "radix": 16}):
        with pytest.raises(capi.NlseError) as ei:
            Batch(cfgs, tuning)
        assert ei.value.status == capi.NLSE_EUNSUPPORTED
    with pytest.raises(capi.NlseError) as ei:
        Batch(mixed_beams((512,)), {"threads": 128, "radix": 8})
    assert ei.value.status == capi.NLSE_EUNSUPPORTED


def test_graph_replay_equals_eager_steps():
    cfgs = mixed_beams((512, 1024, 256))
    fields = [beams.make_field(c).astype(np.complex64) for c in cfgs]
    with Batch(cfgs) as a, Batch(cfgs) as b:
        for i, U in enumerate(fields):
            a.load(i, U)
            b.load(i, U)
        a.step(30)
        b.capture(10)
        for _ in range(3):
            b.replay()
        assert b.status() == capi.NLSE_OK and b.steps_taken == 30
        for i in range(len(cfgs)):
            assert np.array_equal(a.field(i), b.field(i))


def test_batched_beam_matches_oracle():
    cfgs = mixed_beams((256, 512))
    fields = [beams.make_field(c).astype(np.complex64) for c in cfgs]
    with Batch(cfgs) as b:
        for i, U in enumerate(fields):
            b.load(i, U)
        b.step(20)
        for i, c in enumerate(cfgs):
            ref, pw, _ = oracle.march(fields[i].astype(np.complex128), c, 20)
            U = b.field(i).astype(np.complex128)
            assert np.linalg.norm(U - ref) / np.linalg.norm(ref) < 2e-5
            assert abs(b.power(i) / pw[-1] - 1) < 1e-5


def test_missing_completion_times_out_and_context_survives():
    """A work item that never reports completion: the waits on it run out
    (50 ms), the launch stops, the status says NLSE_ETIMEOUT, and the next batch
    on the same device runs normally."""
    cfgs = mixed_beams((512, 256))
    fields = [beams.make_field(c).astype(np.complex64) for c in cfgs]
    with Batch(cfgs, {"timeout_ms": 50, "debug_skip_item": 3}) as b:
        for i, U in enumerate(fields):
            b.load(i, U)
        b.step(5)
        assert b.status() == capi.NLSE_ETIMEOUT
        assert b.status() == capi.NLSE_OK  # cleared
    with Batch(cfgs) as b:
        for i, U in enumerate(fields):
            b.load(i, U)
        b.step(5)
        assert b.status() == capi.NLSE_OK
        assert np.array_equal(b.field(1), single(cfgs[1], fields[1], 5))


def test_batch_rejects_unsupported_inputs():
    cfgs = mixed_beams((512,))
    bad = [dict(cfgs[0], n=128)]
    with pytest.raises(capi.NlseError) as ei:
        Batch(bad)
    assert ei.value.status == capi.NLSE_EUNSUPPORTED
    with pytest.raises(capi.NlseError) as ei:
        Batch(cfgs, {"threads": 384})
    assert ei.value.status == capi.NLSE_EINVAL
    with pytest.raises(capi.NlseError) as ei:
        Batch(cfgs, {"radix": 4})
    assert ei.value.status == capi.NLSE_EINVAL


def test_autotuner_picks_a_valid_shape(tmp_path):
    from paper_2306_15678_gb300 import tune
    cfgs = mixed_beams((512, 1024))
    t = tune.tune_batch(cfgs, steps=3, path=str(tmp_path / "t.json"))
    assert t["threads"] in (128, 256, 512) and t["radix"] in (16, 8)
    assert tune.tune_batch(cfgs, path=str(tmp_path / "t.json")) == t  # cached
    c = tune.tune_grid(configs.scaled(configs.cfg_dense_fp32(), 1024), "fp32", steps=3,
                       path=str(tmp_path / "t.json"))
    assert c in tune.TILE_CODES
