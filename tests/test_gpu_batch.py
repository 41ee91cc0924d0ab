"""Batches (many independent cartograms as parallel branches of one CUDA-graph launch) and
the device-side outer iteration, through the C-ABI. A batch runs the same kernels with
the same arithmetic as each context alone, so step counts must agree exactly with single
runs and vertices to the run-to-run rounding of the rasteriser's FP64 atomic sums (whose
order varies); a failing context must not disturb the others."""
import numpy as np
import pytest

import paper_1802_07625_gb300 as P
from paper_1802_07625_gb300 import synth

pytestmark = pytest.mark.gpu


def _maps():
    return [
        ("voronoi64", synth.make_workload("voronoi16_64"), 1.0, dict(precision="fp64")),
        ("voronoi128", synth.make_workload("voronoi16_64", L=128, n=40), 1.0, dict(precision="mixed")),
        ("strips_linear", synth.strip_map(128, 32, [0, 32, 64, 128], [1.0, 3.0, 0.5], spacing=0.6), 4.0,
         dict(precision="mixed", flow="linear")),
        ("clustered256", synth.make_workload("clustered300_512", L=256, n=120), 2.0, dict(precision="mixed")),
    ]


def _tol(kw):
    return 1e-10 if kw.get("precision", "fp64") == "fp64" else 1e-4


def _run_alone(m, blur, kw):
    with P.Cartogram(m.Lx, m.Ly, blur, **kw) as c:
        c.set_map(m)
        st = c.integrate()
        return st, c.vertices(), [c.grid(k) for k in range(c.history_length())]


def test_batch_matches_single_runs():
    maps = _maps()
    alone = [_run_alone(m, b, kw) for _, m, b, kw in maps]
    carts = []
    try:
        for _, m, b, kw in maps:
            c = P.Cartogram(m.Lx, m.Ly, b, **kw)
            c.set_map(m)
            carts.append(c)
        with P.Batch(carts) as batch:
            stats, status = batch.integrate()
            assert status == [P.CG_OK] * len(maps)
            for (name, *_), c, st, (st1, xy1, grids1) in zip(maps, carts, stats, alone):
                assert st.converged and st1.converged, name
                assert (st.iterations, st.steps_accepted, st.steps_rejected) == \
                    (st1.iterations, st1.steps_accepted, st1.steps_rejected), name
                kw = maps[[mm[0] for mm in maps].index(name)][3]
                d = np.max(np.abs(c.vertices() - xy1))
                assert d < _tol(kw), (name, d)
                assert c.history_length() == len(grids1)
                for k, g in enumerate(grids1):
                    assert np.max(np.abs(c.grid(k) - g)) < _tol(kw), (name, k)
            # a second call on converged maps runs no iteration
            stats2, status2 = batch.integrate()
            assert status2 == [P.CG_OK] * len(maps)
            assert all(s.iterations == 0 for s in stats2)
            # after a reset the same (already captured) graph reproduces the first run
            for c in carts:
                c.reset()
            stats3, _ = batch.integrate()
            for (_, _m, _b, kw), c, (_, xy1, _g) in zip(maps, carts, alone):
                assert np.max(np.abs(c.vertices() - xy1)) < _tol(kw)
    finally:
        for c in carts:
            c.close()


def test_batch_frames_match_oracle(orc):
    """Every cartogram of a batch against the FP64 oracle (the batch's independent problems
    are the paper's independent integrations, run side by side): the 64^2 map in FP64
    (1e-9 grid units, identical step counts), the 128^2 map mixed (1e-3), and the first
    128^2 and 256^2 frames of the batched workload in both precisions against the
    oracle's stored converged results."""
    from test_gpu_golden import MIXED_TOL, AREA_TOL, FP64_TOL, golden_map, load_golden
    maps = _maps()[:2]
    refs = [orc.cartogram(m, b, keep_grids=False) for _, m, b, _ in maps]
    frames = []
    for name in ("batch_frame_128", "batch_frame_256"):
        g = load_golden(name)
        frames.append((name, golden_map(name, g["meta"]), g))
    carts = []
    try:
        for _, m, b, kw in maps:
            carts.append(P.Cartogram(m.Lx, m.Ly, b, **kw))
            carts[-1].set_map(m)
        for _, m, g in frames:
            for precision in ("fp64", "mixed"):
                carts.append(P.Cartogram(m.Lx, m.Ly, g["meta"]["blur"], precision=precision))
                carts[-1].set_map(m)
        with P.Batch(carts) as batch:
            stats, status = batch.integrate()
        assert status == [P.CG_OK] * len(carts)
        for (name, m, b, kw), ref, c, st in zip(maps, refs, carts, stats):
            assert ref.converged and st.converged and st.iterations == ref.iterations, name
            if kw["precision"] == "fp64":
                assert (st.steps_accepted, st.steps_rejected) == (ref.steps_accepted, ref.steps_rejected)
            tol = FP64_TOL if kw["precision"] == "fp64" else MIXED_TOL
            assert np.max(np.abs(c.vertices() - ref.xy)) < tol, name
            assert np.max(np.abs(c.area_errors() - ref.err)) < (FP64_TOL if tol == FP64_TOL else AREA_TOL)
        k = len(maps)
        for name, m, g in frames:
            for precision in ("fp64", "mixed"):
                c, st = carts[k], stats[k]
                k += 1
                meta = g["meta"]
                assert st.converged and st.iterations == meta["iterations"], (name, precision)
                xy = c.vertices()[g["vertex_index"]]
                if precision == "fp64":
                    assert (st.steps_accepted, st.steps_rejected) == \
                        (meta["steps_accepted"], meta["steps_rejected"]), name
                    assert np.max(np.abs(xy - g["xy"])) < FP64_TOL, name
                    assert np.max(np.abs(c.area_errors() - g["err"])) < FP64_TOL, name
                else:
                    assert np.max(np.abs(xy - g["xy"])) < MIXED_TOL, name
                    assert np.max(np.abs(c.area_errors() - g["err"])) < AREA_TOL, name
    finally:
        for c in carts:
            c.close()


def test_batch_reports_each_contexts_failure():
    m = synth.make_workload("voronoi16_64")
    good = P.Cartogram(m.Lx, m.Ly, 1.0, precision="mixed")
    bad = P.Cartogram(m.Lx, m.Ly, 1.0, precision="mixed", max_steps=3, autotune=0)
    tight = P.Cartogram(m.Lx, m.Ly, 1.0, precision="mixed", max_iter=2)
    try:
        for c in (good, bad, tight):
            c.set_map(m)
        with P.Batch([good, bad, tight]) as batch:
            stats, status = batch.integrate(check=False)
        assert status == [P.CG_OK, P.CG_ESTEPFAIL, P.CG_ENOCONVERGE]
        assert stats[0].converged
        assert np.array_equal(bad.vertices(), m.xy)  # a failed integration maps nothing
        assert tight.history_length() == 2
        with pytest.raises(P.CartogramError):
            with P.Batch([good, bad]) as b2:
                bad.reset()
                b2.integrate()
    finally:
        for c in (good, bad, tight):
            c.close()


def test_batch_resumes_when_history_slots_run_out():
    # the 512^2 clustered map needs ~190 iterations: the device loop stops every time its
    # history slots (allocated in chunks) run out, and the host adds slots and relaunches
    big = synth.make_workload("clustered300_512")
    small = synth.make_workload("voronoi16_64")
    st_alone, xy_alone, _ = _run_alone(big, 2.0, dict(precision="mixed"))
    a = P.Cartogram(big.Lx, big.Ly, 2.0, precision="mixed")
    b = P.Cartogram(small.Lx, small.Ly, 1.0, precision="fp64")
    try:
        a.set_map(big)
        b.set_map(small)
        with P.Batch([a, b]) as batch:
            stats, status = batch.integrate()
        assert status == [P.CG_OK, P.CG_OK]
        assert stats[0].iterations == st_alone.iterations > 64
        assert np.max(np.abs(a.vertices() - xy_alone)) < 1e-4
        assert a.history_length() == st_alone.iterations
    finally:
        a.close()
        b.close()


def test_batch_rejects_bad_groups():
    m = synth.make_workload("voronoi16_64")
    c = P.Cartogram(m.Lx, m.Ly, 1.0)
    try:
        with pytest.raises(P.CartogramError):
            P.cartogram_batch_create([c.ctx, c.ctx])
        with pytest.raises(P.CartogramError):
            P.cartogram_batch_create([])
        with P.Batch([c]) as batch:  # no map yet
            stats, status = batch.integrate(check=False)
            assert status == [P.CG_ESTATE]
    finally:
        c.close()


def test_batched_frames_workload_converges():
    # the batched workload's recipe at reduced size: 6 frames from {128, 256} (on a 64^2
    # grid the 300 regions would be ~8 cells^2, below what the grid resolves)
    frames = synth.make_batch(frames=6, sizes=(128, 256))
    carts = [P.Cartogram(f.Lx, f.Ly, synth.BATCH["blur"], precision="mixed") for f in frames]
    try:
        for c, f in zip(carts, frames):
            c.set_map(f)
        with P.Batch(carts) as batch:
            stats, status = batch.integrate()
        assert status == [P.CG_OK] * len(frames)
        for c, f, st in zip(carts, frames, stats):
            assert st.converged and st.max_area_error < 0.01
            assert np.max(np.abs(c.area_errors())) < 0.01
    finally:
        for c in carts:
            c.close()
