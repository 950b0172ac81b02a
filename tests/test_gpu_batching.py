"""Batched, serving-style execution: kernel variants, persistent launches,
CUDA-graph replay, the autotuner, uneven batches, and failure reporting.

Every projector variant computes each ray identically, so projections are
bit-identical across projector variants and launch modes.  Adjoint variants
sum each voxel's angles in the same order but place the fixed-point origin of
the detector coordinate at a different voxel (the tile corner; the mirror
variants derive a voxel's image from the voxel's own position), so the FP32
weights round differently: gradients agree to FP32 rounding.  The objective
does not involve the adjoint and is bit-identical.  Graph replay and
persistent launches are bit-identical to their counterparts; an uneven batch
reproduces each slice solved on its own exactly.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2202_08627_gb300 import inputs
from tests.problems import gpu_geometry, measured, oracle_geometry, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


SHAPES = [(64, 90, 96, 5), (37, 23, 61, 5), (128, 180, 192, 5), (20, 7, 131, 5)]


def _uneven():
    probs = []
    for i, sh in enumerate(SHAPES):
        spec = inputs.make_slice(30 + i, *sh)
        geom = oracle_geometry(spec)
        probs.append((spec, geom, measured(spec, geom)))
    return probs


def _eval(G, xs, meas):
    from paper_2202_08627_gb300 import ei
    S = torch.zeros(G.n_slices, dtype=torch.float64, device="cuda")
    grad = G.empty("vol")
    ei.ei_objective_grad(G, G.pack_volume(xs), meas, S, grad)
    proj = G.empty("proj")
    ei.ei_project(G, G.pack_volume(xs), proj)
    torch.cuda.synchronize()
    return S.cpu().numpy(), grad.cpu().numpy(), proj.cpu().numpy()


def test_every_variant_agrees():
    from paper_2202_08627_gb300 import ei
    probs = _uneven()
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    m = G.pack_meas(meas)
    xs = [sp.truth * 0.9 for sp in specs]
    per_adj = {}
    for a in range(ei.N_ADJ_VARIANTS):
        for f in range(ei.N_FWD_VARIANTS):
            for pers in (0, 1, 2):               # per item, persistent, SM-chunked persistent
                ei.ei_set_variant(G, f, a, pers)
                assert ei.ei_get_variant(G) == (f, a, pers)
                S, grad, proj = _eval(G, xs, m)
                if a not in per_adj:
                    per_adj[a] = (S, grad, proj)
                # same adjoint variant: bit-identical whatever the projector or launch mode
                np.testing.assert_array_equal(S, per_adj[a][0], err_msg=str((f, a, pers)))
                np.testing.assert_array_equal(grad, per_adj[a][1], err_msg=str((f, a, pers)))
                # every projector variant: bit-identical projections
                np.testing.assert_array_equal(proj, per_adj[0][2], err_msg=str((f, a, pers)))
    S0, g0, _ = per_adj[0]
    # variants 11-13 read mirror-interleaved gradient rows with paired FMAs:
    # the same sums as 8-10 in the same order
    for a in (11, 12, 13):
        np.testing.assert_array_equal(per_adj[a][1], per_adj[a - 3][1], err_msg=str(a))
    for a in range(1, ei.N_ADJ_VARIANTS):
        S, g, _ = per_adj[a]
        np.testing.assert_array_equal(S, S0)
        for sl in G.slices:
            blk = slice(sl.vol_offset, sl.vol_offset + sl.vol_count)
            for c in range(3):
                assert rel_l2(g[blk, c], g0[blk, c]) <= 1e-6, (a, c)


def test_staged_projector_equals_global_loads_on_staged_slices():
    """Projector variant 13 stages the rows of most blocks of these slices in
    shared memory (a CPU model of its windows stages 86% of the 256^2
    slice's blocks); the rest (angles mixing row- and column-first rays) load
    from global memory.  Its projections, the objective and the gradient
    equal variant 12's bit for bit, with three channels and linked, in every
    launch mode."""
    from paper_2202_08627_gb300 import ei
    shapes = [(256, 720, 384, 5), (200, 361, 301, 5), (96, 1800, 160, 5)]
    probs = []
    for i, sh in enumerate(shapes):
        spec = inputs.make_slice(70 + i, *sh)
        geom = oracle_geometry(spec)
        probs.append((spec, geom, measured(spec, geom)))
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    m = G.pack_meas(meas)
    xs = [sp.truth * 0.9 for sp in specs]
    for gamma in (0.0, 5e-7):
        ei.ei_set_linked(G, gamma)
        ref = None
        for f, pers in ((12, 0), (13, 0), (13, 1)):
            ei.ei_set_variant(G, f, 8, pers)
            S, grad, proj = _eval(G, xs, m)
            fwd = G.empty("meas")
            ei.ei_forward(G, G.pack_volume(xs), fwd)
            torch.cuda.synchronize()
            got = (S, grad, proj, fwd.cpu().numpy())
            if ref is None:
                ref = got
                continue
            for name, a, b in zip(("S", "grad", "proj", "forward"), got, ref):
                np.testing.assert_array_equal(a, b, err_msg="%s gamma=%g variant=%d mode=%d"
                                              % (name, gamma, f, pers))
    ei.ei_set_linked(G, 0.0)


def test_mirror_interleaved_adjoint_equals_pair_packed():
    """Adjoint variants 11-13 read gradient rows whose entry j holds pixel j
    and its mirror pixel n_det - 1 - j (written by the IC kernels and, for
    ei_backproject, by k_pack_sino, for the single-shot starts by their row
    filter) and advance a voxel and its point mirror with one paired FP32 FMA;
    variants 8-10 read the pair-packed rows with scalar FMAs in the same
    order.  Gradients (three channels and linked), plain back-projections and
    both single-shot starts are equal bit for bit, and switching the layout
    back and forth leaves nothing stale."""
    from paper_2202_08627_gb300 import ei
    probs = _uneven()
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    m = G.pack_meas(meas)
    xs = [sp.truth * 0.9 for sp in specs]
    rng = np.random.default_rng(5)
    sino = torch.from_numpy(rng.standard_normal((G.sino4_count, 4)).astype(np.float32)).cuda()
    first = {}
    for gamma in (0.0, 5e-7):
        ei.ei_set_linked(G, gamma)
        for a in (8, 11, 9, 12, 10, 13, 8):
            ei.ei_set_variant(G, 12, a, 0)
            S, grad, _ = _eval(G, xs, m)
            bp = G.empty("vol")
            ei.ei_backproject(G, sino, bp)
            fbp = G.empty("vol")
            ei.ei_single_shot_fbp(G, m, fbp)
            eq3 = G.empty("vol")
            ei.ei_single_shot_eq3(G, m, 2, 5e-7, eq3)
            torch.cuda.synchronize()
            got = (S, grad, bp.cpu().numpy(), fbp.cpu().numpy(), eq3.cpu().numpy())
            key = (gamma, a if a < 11 else a - 3)
            if key not in first:
                first[key] = got
                continue
            for name, x, y in zip(("S", "grad", "backproject", "single-shot FBP", "Eq. 3 single shot"),
                                  got, first[key]):
                np.testing.assert_array_equal(x, y, err_msg="%s gamma=%g variant=%d" % (name, gamma, a))
    ei.ei_set_linked(G, 0.0)


def test_graph_replay_equals_eager_rounds():
    from paper_2202_08627_gb300 import ei
    probs = _uneven()
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    m = G.pack_meas(meas)
    out = {}
    for use_graph in (False, True):
        vol = G.empty("vol")
        rep = ei.ei_reconstruct(G, m, vol, tol=0.0, max_iter=12, use_graph=use_graph)
        out[use_graph] = (vol.cpu().numpy(), rep.f_final.copy(), rep.iterations.copy())
    np.testing.assert_array_equal(out[False][0], out[True][0])
    np.testing.assert_array_equal(out[False][1], out[True][1])
    np.testing.assert_array_equal(out[False][2], out[True][2])


def test_uneven_batch_solve_equals_single_slice_solves():
    from paper_2202_08627_gb300 import ei
    probs = _uneven()
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    vol = G.empty("vol")
    rep = ei.ei_reconstruct(G, G.pack_meas(meas), vol, tol=1e-7, max_iter=15)
    batch = G.unpack_volume(vol)
    for i, (spec, geom, s_exp) in enumerate(probs):
        G1 = gpu_geometry([spec], [geom])
        v1 = G1.empty("vol")
        r1 = ei.ei_reconstruct(G1, G1.pack_meas([s_exp]), v1, tol=1e-7, max_iter=15)
        assert r1.iterations[0] == rep.iterations[i]
        assert r1.f_final[0] == rep.f_final[i]
        np.testing.assert_array_equal(G1.unpack_volume(v1)[0], batch[i])


def test_autotune_selects_and_caches(tmp_path, monkeypatch):
    from paper_2202_08627_gb300 import ei
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("EI_TUNE_CACHE", str(cache))
    probs = _uneven()
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    m = G.pack_meas(meas)
    xs = [sp.truth * 0.9 for sp in specs]
    ref = _eval(G, xs, m)
    choice = ei.ei_autotune(G, force=True)
    assert 0 <= choice[0] < ei.N_FWD_VARIANTS and 0 <= choice[1] < ei.N_ADJ_VARIANTS
    lines = cache.read_text().split("\n")
    assert len([ln for ln in lines if ln.strip()]) == 1
    # another geometry of the same shapes reads the cached choice back
    G2 = gpu_geometry(list(specs), list(geoms))
    assert ei.ei_autotune(G2) == choice
    assert len([ln for ln in cache.read_text().split("\n") if ln.strip()]) == 1
    S, grad, proj = _eval(G, xs, m)
    np.testing.assert_array_equal(proj, ref[2])
    np.testing.assert_allclose(S, ref[0], rtol=1e-12)
    for c in range(3):
        assert rel_l2(grad[:, c], ref[1][:, c]) <= 1e-6


def test_failures_are_reported_per_slice():
    """A NaN in one slice's data and a start outside the model's domain in
    another are reported for those slices; the remaining slice converges."""
    from paper_2202_08627_gb300 import ei
    probs = _uneven()[:3]
    specs, geoms, meas = zip(*probs)
    meas = [m.copy() for m in meas]
    meas[0][0, 0, 0] = np.nan
    G = gpu_geometry(list(specs), list(geoms))
    x0 = [np.zeros((3, sp.n, sp.n)) for sp in specs]
    x0[1][2] = -50.0                   # scatter far below zero: V <= 0.01 w^2
    vol = G.pack_volume(x0)
    rep = ei.ei_reconstruct(G, G.pack_meas(meas), vol, tol=1e-6, max_iter=30,
                            raise_on_error=False)
    assert rep.status[0] == ei.EI_ERR_NONFINITE
    assert rep.status[1] == ei.EI_ERR_NONFINITE
    assert rep.status[2] == ei.EI_OK and rep.iterations[2] > 0
    assert rep.return_status == ei.EI_ERR_NONFINITE


def test_linesearch_failure_is_reported():
    """Armijo with c1 = 0.9999 asks a step to achieve almost the whole linear
    decrease, which a locally convex cost never allows: with two trials the
    line search must fail and be reported as EI_ERR_LINESEARCH (not hang)."""
    from paper_2202_08627_gb300 import ei
    probs = _uneven()[:2]
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    vol = G.empty("vol")
    rep = ei.ei_reconstruct(G, G.pack_meas(meas), vol, tol=0.0, max_iter=20, c1=0.9999,
                            max_trials=2, raise_on_error=False)
    statuses = set(rep.status.tolist())
    assert ei.EI_ERR_LINESEARCH in statuses and statuses <= {ei.EI_OK, ei.EI_ERR_LINESEARCH}
    assert rep.return_status == ei.EI_ERR_LINESEARCH
