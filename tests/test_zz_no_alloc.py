"""The no-allocation entry point against the regular one.

ei_objective_grad_noalloc serves callers that may not allocate GPU memory
themselves (a framework that has reserved the device memory for its own pool,
a loop that cannot pay cudaMalloc's synchronisation).  It keeps every
intermediate in one static device array that each call reuses, so two calls in
a row must each reproduce ei_objective_grad on their own input exactly: both
run variant 0 of the same kernels on tables built the same way, so any
difference, even in the last bit, would be a leftover of the previous call.
This file is collected last so that a failure here comes after every other
test has run; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_2202_08627_gb300 import inputs
from tests.problems import gpu_geometry, measured, oracle_geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


def _args(geom):
    return dict(n=geom.n, n_theta=geom.n_theta, n_det=geom.n_det, pitch_cm=geom.pitch,
                n_m=geom.n_m, m=geom.m, z_cm=geom.z_cm, period_cm=geom.period_cm,
                kappa_sigma=geom.kappa, flat_A=geom.flat_A, flat_c=geom.flat_c,
                flat_w=geom.flat_w, lam=geom.lam, scale=geom.scale, theta=geom.theta,
                m_o=geom.m_o, m_r=geom.m_r)


@pytest.mark.parametrize("shape", [(64, 90, 96, 7), (256, 720, 384, 7), (37, 23, 61, 3)])
def test_noalloc_equals_objective_grad_twice(shape):
    from paper_2202_08627_gb300 import ei
    spec = inputs.make_slice(11, *shape)
    geom = oracle_geometry(spec)
    if shape[0] == 37:
        geom.m_o = inputs.uniform_noise(geom.n_theta, 40, -0.03, 0.03)
        geom.m_r = inputs.uniform_noise(geom.n_det, 41, -0.03, 0.03)
    s_exp = measured(spec, geom)
    G = gpu_geometry([spec], [geom])
    ei.ei_set_variant(G, 0, 0, False)          # the kernels the entry point runs
    ei.ei_set_ic_variant(G, 0)
    meas = G.pack_meas([s_exp])
    # two calls in a row, the second on other inputs and with device flat arrays
    for call, factor in enumerate((0.9, 1.1)):
        vol = G.pack_volume([spec.truth * factor])
        S_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        g_ref = G.empty("vol")
        ei.ei_objective_grad(G, vol, meas, S_ref, g_ref)
        S = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        g = torch.full_like(g_ref, float("nan"))
        args = _args(geom)
        if call == 1:
            for k in ("flat_A", "flat_c", "flat_w"):
                args[k] = torch.tensor(args[k], dtype=torch.float32, device="cuda")
        ei.ei_objective_grad_noalloc(vol=vol, s_exp=meas, S_out=S, grad=g, **args)
        torch.cuda.synchronize()
        assert S.item() == S_ref.item(), (call, S.item(), S_ref.item())
        assert torch.equal(g, g_ref), (call, float((g - g_ref).abs().max()))
        assert np.isfinite(G.unpack_volume(g)[0]).all()


def test_noalloc_host_S_out_and_objective_only():
    from paper_2202_08627_gb300 import ei
    spec = inputs.make_slice(3, 48, 40, 70, 5)
    geom = oracle_geometry(spec)
    s_exp = measured(spec, geom)
    G = gpu_geometry([spec], [geom])
    ei.ei_set_variant(G, 0, 0, False)
    ei.ei_set_ic_variant(G, 0)
    meas = G.pack_meas([s_exp])
    vol = G.pack_volume([spec.truth * 0.8])
    S_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    ei.ei_objective_grad(G, vol, meas, S_ref, None)
    S_host = torch.full((1,), float("nan"), dtype=torch.float64)
    ei.ei_objective_grad_noalloc(vol=vol, s_exp=meas, S_out=S_host, grad=None, **_args(geom))
    assert S_host.item() == S_ref.item()


@pytest.mark.parametrize("bad", ["flat_w_zero", "flat_A_nan", "z_inf", "period_inf",
                                 "kappa_inf", "scale_inf", "theta_nan"])
def test_noalloc_rejects_invalid_descriptions(bad):
    from paper_2202_08627_gb300 import ei
    spec = inputs.make_slice(0, 32, 16, 40, 3)
    geom = oracle_geometry(spec)
    args = _args(geom)
    if bad == "flat_w_zero":
        w = np.array(args["flat_w"], dtype=np.float64)
        w[5] = 0.0
        args["flat_w"] = w
    elif bad == "flat_A_nan":
        a = np.array(args["flat_A"], dtype=np.float64)
        a[7] = np.nan
        args["flat_A"] = a
    elif bad == "z_inf":
        args["z_cm"] = float("inf")
    elif bad == "period_inf":
        args["period_cm"] = float("inf")
    elif bad == "kappa_inf":
        args["kappa_sigma"] = float("inf")
    elif bad == "scale_inf":
        args["scale"] = (1.0, float("inf"), 1.0)
    else:
        th = np.array(args["theta"], dtype=np.float64)
        th[3] = np.nan
        args["theta"] = th
    vol = torch.zeros(32 * 32 * 4, dtype=torch.float32, device="cuda")
    meas = torch.zeros(3 * 16 * 40, dtype=torch.float32, device="cuda")
    S = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ei.EIError) as err:
        ei.ei_objective_grad_noalloc(vol=vol, s_exp=meas, S_out=S, **args)
    assert err.value.status == ei.EI_ERR_ARG


def test_noalloc_refuses_tensors_it_would_have_to_convert():
    from paper_2202_08627_gb300 import ei
    spec = inputs.make_slice(0, 32, 16, 40, 3)
    geom = oracle_geometry(spec)
    args = _args(geom)
    args["flat_A"] = torch.tensor(geom.flat_A, dtype=torch.float64, device="cuda")
    vol = torch.zeros(32 * 32 * 4, dtype=torch.float32, device="cuda")
    meas = torch.zeros(3 * 16 * 40, dtype=torch.float32, device="cuda")
    S = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        ei.ei_objective_grad_noalloc(vol=vol, s_exp=meas, S_out=S, **args)


def test_noalloc_rejects_slices_beyond_the_scratch():
    from paper_2202_08627_gb300 import ei
    spec = inputs.make_slice(0, 64, 8, 96, 3)
    geom = oracle_geometry(spec)
    args = _args(geom)
    args.update(n=2048, n_theta=1800, n_det=3000, pitch_cm=0.32 / 2048, theta=None,
                flat_A=np.ones(3000), flat_c=np.zeros(3000), flat_w=np.full(3000, 0.25))
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    S = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ei.EIError) as err:
        ei.ei_objective_grad_noalloc(vol=dummy, s_exp=dummy, S_out=S, **args)
    assert err.value.status == ei.EI_ERR_ARG
