"""Parity at the benchmark's full size, in the configuration bench.py times.

The 256-slice uneven workload (1024^2 and 512^2 slices, 1800 angles,
1024-1536 pixels, M = 7) runs through ei_objective_grad with the autotuned
kernel variants.  Two sampled slices — one 1024^2 and one 512^2 — get measured
ICs made by the oracle (analytic projections, the oracle's IC model, Poisson
noise); their objective and full gradient are compared with the FP64 oracle.
The other slices carry zero data, which is still a valid problem; their
objectives must be finite.
"""
import numpy as np
import pytest

import oracle
from paper_2202_08627_gb300 import inputs, workloads
from tests.problems import rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


def test_full_size_sampled_slices_match_oracle(tmp_path, monkeypatch):
    from paper_2202_08627_gb300 import ei
    monkeypatch.setenv("EI_TUNE_CACHE", str(tmp_path / "tune.txt"))
    wl = workloads.uneven1024()
    flats = [inputs.flat_ic(1000 + s, nd) for s, (n, nth, nd) in enumerate(wl.slices)]
    thetas = [inputs.angles(nth) for (n, nth, nd) in wl.slices]
    m = inputs.mask_positions(wl.n_m)
    G = ei.ei_setup_geometry(
        n_m=wl.n_m, m=m, z_cm=inputs.Z_CM, period_cm=inputs.PERIOD_CM, kappa_sigma=inputs.KAPPA,
        flat_A=np.concatenate([f[0] for f in flats]), flat_c=np.concatenate([f[1] for f in flats]),
        flat_w=np.concatenate([f[2] for f in flats]), lam=(inputs.LAMBDA,) * 3, scale=inputs.SCALE,
        per_slice=wl.per_slice(), theta=np.concatenate(thetas))
    ei.ei_autotune(G)
    sampled = [0, 1]                                    # a 1024^2 and a 512^2 slice
    meas = G.empty("meas")
    vol = G.empty("vol")
    refs = {}
    for s in sampled:
        n, nth, nd = wl.slices[s]
        spec = inputs.make_slice(2000 + s, n, nth, nd, wl.n_m, flat_seed=1000 + s)
        og = oracle.Geometry(n=n, n_theta=nth, n_det=nd, pitch=spec.pitch, theta=spec.theta, m=m,
                             z_cm=inputs.Z_CM, period_cm=inputs.PERIOD_CM, kappa=inputs.KAPPA,
                             flat_A=spec.flat_A, flat_c=spec.flat_c, flat_w=spec.flat_w)
        s_exp = inputs.poisson_noise(oracle.ic_model(spec.P_exact, og), spec.seed)
        sl = G.slices[s]
        blk = np.zeros((wl.n_m, nth, sl.n_dp), np.float32)
        blk[:, :, :nd] = s_exp
        meas[sl.meas_offset:sl.meas_offset + sl.meas_count] = torch.from_numpy(blk.ravel()).cuda()
        x = spec.truth * 0.9
        v = np.zeros((n * n, 4), np.float32)
        v[:, :3] = x.reshape(3, -1).T
        vol[sl.vol_offset:sl.vol_offset + sl.vol_count] = torch.from_numpy(v).cuda()
        refs[s] = oracle.objective_grad(x, s_exp, og)
    S = torch.zeros(G.n_slices, dtype=torch.float64, device="cuda")
    grad = G.empty("vol")
    ei.ei_objective_grad(G, vol, meas, S, grad)
    torch.cuda.synchronize()
    Sh = S.cpu().numpy()
    assert np.all(np.isfinite(Sh))
    g_all = grad.cpu().numpy()
    for s in sampled:
        S_ref, g_ref = refs[s]
        assert abs(Sh[s] - S_ref) <= 1e-5 * abs(S_ref), (s, Sh[s], S_ref)
        sl = G.slices[s]
        g = g_all[sl.vol_offset:sl.vol_offset + sl.vol_count, :3].T.reshape(3, sl.n, sl.n)
        for c in range(3):
            assert rel_l2(g[c], g_ref[c]) <= 1e-4, (s, c, rel_l2(g[c], g_ref[c]))
