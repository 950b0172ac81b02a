"""The fused IC kernel's two variants: one block per sinogram row (0) and
persistent blocks streaming rows through shared memory with bulk
asynchronous copies (1).  Both evaluate Eq. 2, the Eq. 5 residual and its
gradient per pixel; they differ in the exponential's evaluation and summation
grouping, so they agree to FP32 rounding, and each matches the FP64 oracle
within the path's tolerances (objective 1e-5 relative, gradient 1e-4 relative
L2)."""
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


def _problems(shapes, seed0):
    out = []
    for i, sh in enumerate(shapes):
        spec = inputs.make_slice(seed0 + i, *sh)
        geom = oracle_geometry(spec)
        out.append((spec, geom, measured(spec, geom)))
    return out


def _evaluate(G, xs, meas):
    from paper_2202_08627_gb300 import ei
    S = torch.zeros(G.n_slices, dtype=torch.float64, device="cuda")
    grad = G.empty("vol")
    vol = G.pack_volume(xs)
    ei.ei_objective_grad(G, vol, meas, S, grad)
    s_mod = G.empty("meas")
    ei.ei_forward(G, vol, s_mod)
    torch.cuda.synchronize()
    return S.cpu().numpy(), G.unpack_volume(grad), G.unpack_meas(s_mod)


def _check_oracle(probs, xs, S, grads, s_mods):
    for (spec, geom, s_exp), x, Sg, g, sm in zip(probs, xs, S, grads, s_mods):
        So, go = oracle.objective_grad(x, s_exp, geom)
        assert abs(Sg - So) <= 1e-5 * abs(So), (spec.n, spec.n_det, Sg, So)
        for c in range(3):
            assert rel_l2(g[c], go[c]) <= 1e-4, (spec.n, spec.n_det, c, rel_l2(g[c], go[c]))
        assert rel_l2(sm, oracle.forward(x, geom)) <= 1e-5


SHAPES = [(64, 90, 96, 5), (37, 23, 61, 5), (128, 180, 192, 5), (20, 7, 131, 5)]


def test_variants_agree_on_an_uneven_batch():
    from paper_2202_08627_gb300 import ei
    probs = _problems(SHAPES, 60)
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    assert ei.ei_get_ic_variant(G) == 1            # these rows fit the bulk-copy variant
    m = G.pack_meas(meas)
    xs = [sp.truth * 0.9 for sp in specs]
    res = {}
    for v in (1, 0):
        ei.ei_set_ic_variant(G, v)
        assert ei.ei_get_ic_variant(G) == v
        res[v] = _evaluate(G, xs, m)
        _check_oracle(probs, xs, *res[v])
    np.testing.assert_allclose(res[1][0], res[0][0], rtol=1e-6)
    for g1, g0 in zip(res[1][1], res[0][1]):
        for c in range(3):
            assert rel_l2(g1[c], g0[c]) <= 1e-5
    for s1, s0 in zip(res[1][2], res[0][2]):
        assert rel_l2(s1, s0) <= 1e-6


def test_bulk_copy_rows_wider_than_the_block():
    """Rows of 2400 pixels: 600 groups of 4 for at most 512 threads, so
    threads loop within a row; M = 3 keeps both row buffers in shared memory."""
    from paper_2202_08627_gb300 import ei
    probs = _problems([(32, 12, 2400, 3), (24, 9, 2100, 3)], 80)
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    assert ei.ei_get_ic_variant(G) == 1
    xs = [sp.truth * 1.1 for sp in specs]
    _check_oracle(probs, xs, *_evaluate(G, xs, G.pack_meas(meas)))


def test_rows_too_wide_for_the_buffers_use_one_block_per_row():
    from paper_2202_08627_gb300 import ei
    probs = _problems([(32, 8, 4000, 7)], 90)
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    assert ei.ei_get_ic_variant(G) == 0
    with pytest.raises(ei.EIError):
        ei.ei_set_ic_variant(G, 1)
    assert ei.ei_get_ic_variant(G) == 0
    xs = [sp.truth * 0.8 for sp in specs]
    _check_oracle(probs, xs, *_evaluate(G, xs, G.pack_meas(meas)))


def test_solves_agree_across_variants():
    """The batched L-BFGS (per-slice active masks skip converged slices' rows)
    reaches the same objective with either variant."""
    from paper_2202_08627_gb300 import ei
    probs = _problems(SHAPES, 100)
    specs, geoms, meas = zip(*probs)
    G = gpu_geometry(list(specs), list(geoms))
    m = G.pack_meas(meas)
    f = {}
    for v in (1, 0):
        ei.ei_set_ic_variant(G, v)
        vol = G.empty("vol")
        rep = ei.ei_reconstruct(G, m, vol, tol=1e-6, max_iter=60)
        f[v] = rep.f_final
    np.testing.assert_allclose(f[1], f[0], rtol=1e-4)
