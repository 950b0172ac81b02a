"""Checkpoint / resume of the solver: a solve stopped at max_iter, saved,
loaded into a fresh geometry and resumed reaches exactly (bit for bit) the
iterate of one uninterrupted solve; mismatched checkpoints are rejected."""
import numpy as np
import pytest

from paper_2202_08627_gb300 import inputs
from tests.problems import gpu_geometry, measured, oracle_geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(48, 40, 64, 5), (37, 23, 61, 5), (20, 7, 131, 5)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


def _problem(seed0, linked=False):
    specs = [inputs.make_slice(seed0 + i, *sh) for i, sh in enumerate(SHAPES)]
    geoms = [oracle_geometry(sp) for sp in specs]
    meas = [measured(sp, g) for sp, g in zip(specs, geoms)]
    return specs, geoms, meas


def _geometry(specs, geoms, linked):
    from paper_2202_08627_gb300 import ei
    G = gpu_geometry(specs, geoms)
    if linked:
        ei.ei_set_linked(G, 5e-7)
    return G


@pytest.mark.parametrize("linked", [False, True])
def test_saved_and_resumed_solve_equals_one_solve(linked):
    from paper_2202_08627_gb300 import ei
    specs, geoms, meas = _problem(1500, linked)
    # one solve of 20 iterations
    G = _geometry(specs, geoms, linked)
    m = G.pack_meas(meas)
    vol_a = G.empty("vol")
    rep_a = ei.ei_reconstruct(G, m, vol_a, tol=0.0, max_iter=20)
    # 8 iterations, checkpoint, a fresh geometry, load, resume to 20
    G1 = _geometry(specs, geoms, linked)
    vol_b = G1.empty("vol")
    rep_1 = ei.ei_reconstruct(G1, G1.pack_meas(meas), vol_b, tol=0.0, max_iter=8)
    assert (rep_1.iterations == 8).all()
    state = ei.ei_solver_save(G1)
    assert state.nbytes == ei.ei_solver_state_size(G1)
    G1.close()
    G2 = _geometry(specs, geoms, linked)
    ei.ei_solver_load(G2, state)
    vol_c = G2.empty("vol")
    rep_c = ei.ei_reconstruct(G2, G2.pack_meas(meas), vol_c, tol=0.0, max_iter=20, resume=True)
    torch.cuda.synchronize()
    assert torch.equal(vol_a, vol_c)
    np.testing.assert_array_equal(rep_c.iterations, rep_a.iterations)
    np.testing.assert_array_equal(rep_c.f_final, rep_a.f_final)
    np.testing.assert_array_equal(rep_c.f_initial, rep_a.f_initial)
    # resuming in place, without a save, continues the same way
    G3 = _geometry(specs, geoms, linked)
    vol_d = G3.empty("vol")
    ei.ei_reconstruct(G3, G3.pack_meas(meas), vol_d, tol=0.0, max_iter=12)
    ei.ei_reconstruct(G3, G3.pack_meas(meas), vol_d, tol=0.0, max_iter=20, resume=True)
    torch.cuda.synchronize()
    assert torch.equal(vol_a, vol_d)


def test_mismatched_or_missing_state_is_rejected():
    from paper_2202_08627_gb300 import ei
    specs, geoms, meas = _problem(1600)
    G = _geometry(specs, geoms, False)
    vol = G.empty("vol")
    with pytest.raises(ei.EIError):                       # nothing to resume from
        ei.ei_reconstruct(G, G.pack_meas(meas), vol, tol=0.0, max_iter=5, resume=True)
    with pytest.raises(ei.EIError):                       # nothing to save
        ei.ei_solver_save(G)
    ei.ei_reconstruct(G, G.pack_meas(meas), vol, tol=0.0, max_iter=3)
    state = ei.ei_solver_save(G)
    with pytest.raises(ei.EIError):                       # another lbfgs_m
        ei.ei_solver_load(G, state, lbfgs_m=5)
    Gl = _geometry(specs, geoms, True)                   # another mode
    with pytest.raises(ei.EIError):
        ei.ei_solver_load(Gl, state)
    other = [inputs.make_slice(1700, 32, 20, 40, 5)]      # another geometry
    Go = gpu_geometry(other, [oracle_geometry(other[0])])
    with pytest.raises(ei.EIError):
        ei.ei_solver_load(Go, np.zeros(ei.ei_solver_state_size(Go), np.uint8))
