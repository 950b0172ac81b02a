"""Failure detection on the host: an allocation made to fail at every point of
the geometry's set-up, of the solver's state and of a U-Net's creation leaves
nothing allocated and the library usable; a solve's time budget stops it
between rounds, and a resumed call continues it bit for bit.  Nothing here
faults, traps or stalls the GPU: the failures are host decisions."""
import contextlib
import gc

import numpy as np
import pytest

from paper_2202_08627_gb300 import inputs
from tests.problems import gpu_geometry, measured, oracle_geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(40, 30, 56, 5), (29, 17, 45, 5)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build, ei
    build.build()
    yield
    ei.ei_fail_alloc_after(-1)


@contextlib.contextmanager
def _counting():
    """Objects of earlier tests that the cyclic collector frees would change
    the live count in the middle of a comparison: collect them first and keep
    the collector off while counting."""
    gc.collect()
    gc.disable()
    try:
        yield
    finally:
        gc.enable()


def _problem(seed0):
    specs = [inputs.make_slice(seed0 + i, *sh) for i, sh in enumerate(SHAPES)]
    geoms = [oracle_geometry(sp) for sp in specs]
    meas = [measured(sp, g) for sp, g in zip(specs, geoms)]
    return specs, geoms, meas


def test_setup_frees_everything_when_any_allocation_fails():
    specs, geoms, _ = _problem(1700)
    with _counting():
        _setup_failures(specs, geoms)


def _setup_failures(specs, geoms):
    from paper_2202_08627_gb300 import ei
    base = ei.ei_live_allocations()
    G = gpu_geometry(specs, geoms)
    count = ei.ei_live_allocations() - base
    G.close()
    assert ei.ei_live_allocations() == base
    assert count >= 20
    for k in range(count):
        ei.ei_fail_alloc_after(k)
        with pytest.raises(ei.EIError) as err:
            gpu_geometry(specs, geoms)
        assert err.value.status == ei.EI_ERR_ALLOC, k
        assert ei.ei_fail_alloc_pending() == -1, k          # it fired
        assert ei.ei_live_allocations() == base, k
    ei.ei_fail_alloc_after(count)                           # one past the last: no failure
    G = gpu_geometry(specs, geoms)
    assert ei.ei_fail_alloc_pending() == 0
    ei.ei_fail_alloc_after(-1)
    G.close()
    assert ei.ei_live_allocations() == base


def test_solver_allocation_failure_leaves_the_geometry_usable():
    from paper_2202_08627_gb300 import ei
    specs, geoms, meas = _problem(1710)
    # reference: five iterations on a geometry that never failed
    R = gpu_geometry(specs, geoms)
    vol_ref = R.empty("vol")
    ei.ei_reconstruct(R, R.pack_meas(meas), vol_ref, tol=0.0, max_iter=5)
    R.close()
    G = gpu_geometry(specs, geoms)
    m = G.pack_meas(meas)
    vol = G.empty("vol")
    with _counting():
        base = ei.ei_live_allocations()
        for k in (0, 1, 6, 12):                             # inside the solver's state
            ei.ei_fail_alloc_after(k)
            rep = ei.ei_reconstruct(G, m, vol, tol=0.0, max_iter=5, raise_on_error=False)
            assert rep.return_status == ei.EI_ERR_ALLOC, k
            assert ei.ei_live_allocations() == base, k
        ei.ei_fail_alloc_after(-1)
    vol.zero_()
    rep = ei.ei_reconstruct(G, m, vol, tol=0.0, max_iter=5)
    torch.cuda.synchronize()
    assert (rep.iterations == 5).all()
    assert torch.equal(vol, vol_ref)
    G.close()


def test_unet_creation_frees_everything_when_an_allocation_fails():
    with _counting():
        _unet_failures()


def _unet_failures():
    from paper_2202_08627_gb300 import ei
    base = ei.ei_live_allocations()
    net = ei.UNet(levels=2, base=32, batch=2, height=32, width=32, seed=3)
    count = ei.ei_live_allocations() - base
    net.close()
    assert ei.ei_live_allocations() == base and count > 10
    for k in sorted({0, 1, count // 3, count // 2, count - 1}):
        ei.ei_fail_alloc_after(k)
        with pytest.raises(ei.EIError) as err:
            ei.UNet(levels=2, base=32, batch=2, height=32, width=32, seed=3)
        assert err.value.status == ei.EI_ERR_ALLOC, k
        assert ei.ei_live_allocations() == base, k
    ei.ei_fail_alloc_after(-1)


def test_time_budget_stops_between_rounds_and_resume_continues_exactly():
    from paper_2202_08627_gb300 import ei
    specs, geoms, meas = _problem(1720)
    A = gpu_geometry(specs, geoms)
    vol_a = A.empty("vol")
    rep_a = ei.ei_reconstruct(A, A.pack_meas(meas), vol_a, tol=0.0, max_iter=12)
    # a budget that has run out before the first round: the initial evaluation
    # only, every slice reported as stopped by it
    B = gpu_geometry(specs, geoms)
    m = B.pack_meas(meas)
    vol_b = B.empty("vol")
    rep_b = ei.ei_reconstruct(B, m, vol_b, tol=0.0, max_iter=12, max_seconds=1e-9)
    assert rep_b.return_status == ei.EI_ERR_TIMEOUT
    assert (rep_b.status == ei.EI_ERR_TIMEOUT).all()
    assert (rep_b.iterations == 0).all()
    np.testing.assert_array_equal(rep_b.f_initial, rep_a.f_initial)
    rep_c = ei.ei_reconstruct(B, m, vol_b, tol=0.0, max_iter=12, resume=True)
    torch.cuda.synchronize()
    assert rep_c.return_status == ei.EI_OK
    assert torch.equal(vol_a, vol_b)
    np.testing.assert_array_equal(rep_c.iterations, rep_a.iterations)
    np.testing.assert_array_equal(rep_c.f_final, rep_a.f_final)
    # an ample budget changes nothing
    C = gpu_geometry(specs, geoms)
    vol_c = C.empty("vol")
    rep_d = ei.ei_reconstruct(C, C.pack_meas(meas), vol_c, tol=0.0, max_iter=12, max_seconds=600.0)
    torch.cuda.synchronize()
    assert rep_d.return_status == ei.EI_OK and torch.equal(vol_a, vol_c)
    for bad in (-1.0, float("nan")):
        with pytest.raises(ei.EIError) as err:
            ei.ei_reconstruct(C, C.pack_meas(meas), vol_c, max_seconds=bad)
        assert err.value.status == ei.EI_ERR_ARG
    for G in (A, B, C):
        G.close()
