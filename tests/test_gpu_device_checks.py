"""The debug build with device-side bounds checks (libei_check.so).

The projector and the adjoint index the packed volume copies and the packed
gradient rows through zero margins that the host sizes from closed forms,
with no checks in the regular build.  The check build verifies every such
index on the device and records EI_ERR_DEVICE_CHECK instead of reading out of
bounds.  Here a child process loads the check build and evaluates S and its
gradient for every projector and every adjoint variant on uneven slices (odd
sizes included) and on 1024 x 1024 slices whose margins are the tightest
(n_det = 1024 and 1536), then runs a short solve: no check may fire, and
every result must equal the regular build's bit for bit (the checks change
no arithmetic).  The check build's self-test shows that a failed check is
recorded: a read whose index leaves its logical range, but not its buffer.
"""
import hashlib
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2202_08627_gb300 import inputs
from tests.problems import gpu_geometry, measured, oracle_geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPES = [(64, 90, 96, 5), (37, 23, 61, 5), (20, 7, 131, 5), (1024, 48, 1024, 3), (1024, 40, 1536, 3)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()
    build.build_checked()


def _problems():
    out = []
    for i, sh in enumerate(SHAPES):
        spec = inputs.make_slice(60 + i, *sh)
        geom = oracle_geometry(spec)
        out.append((spec, geom, measured(spec, geom)))
    return out


def _digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _evaluations():
    """{key: (S, digest of grad)} for every projector variant with adjoint 0
    and every adjoint variant with projector 12, per shape (one slice per
    geometry), and the final objectives and iterate of a 4-iteration solve of
    the uneven batch."""
    from paper_2202_08627_gb300 import ei
    results, statuses = {}, []
    probs = _problems()
    for k, (spec, geom, meas) in enumerate(probs):
        G = gpu_geometry([spec], [geom])
        m = G.pack_meas([meas])
        vol = G.pack_volume([spec.truth * 0.9])
        combos = [(f, 0) for f in range(ei.N_FWD_VARIANTS)] + \
                 [(12, a) for a in range(ei.N_ADJ_VARIANTS)]
        for f, a in combos:
            ei.ei_set_variant(G, f, a, False)
            S = torch.zeros(1, dtype=torch.float64)              # host S_out: synchronous,
            g = G.empty("vol")                                  # reports the status word
            rc = ei.load_library().ei_objective_grad(G.handle, vol.data_ptr(), m.data_ptr(),
                                                     S.data_ptr(), g.data_ptr(), None)
            statuses.append(rc)
            results["%d/%d/%d" % (k, f, a)] = (S.numpy().tolist(), _digest(g.cpu().numpy()))
        G.close()
    small = probs[:3]
    G = gpu_geometry([p[0] for p in small], [p[1] for p in small])
    ei.ei_set_variant(G, 12, 8, False)
    vol = G.empty("vol")
    rep = ei.ei_reconstruct(G, G.pack_meas([p[2] for p in small]), vol, tol=0.0, max_iter=4,
                            raise_on_error=False)
    statuses.append(rep.return_status)
    results["solve"] = (rep.f_final.tolist(), _digest(vol.cpu().numpy()))
    G.close()
    return results, statuses


def _child(out_path):
    """Run in a process whose EI_LIBRARY is the check build."""
    from paper_2202_08627_gb300 import ei
    torch.cuda.set_device(0)
    info = {"enabled": ei.ei_device_checks_enabled(), "selftest": ei.ei_selftest_device_check()}
    results, statuses = _evaluations()
    info["statuses"] = statuses
    info["results"] = results
    with open(out_path + ".json", "w") as f:
        json.dump(info, f)


def test_check_build_fires_on_a_bad_index_and_nowhere_else(tmp_path):
    from paper_2202_08627_gb300 import build, ei
    out = str(tmp_path / "check")
    env = dict(os.environ, EI_LIBRARY=build.CHECK_LIB)
    code = "import sys; sys.path.insert(0, %r); import tests.test_gpu_device_checks as t; t._child(%r)" \
        % (ROOT, out)
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    info = json.load(open(out + ".json"))
    assert info["enabled"] is True
    assert info["selftest"] == ei.EI_ERR_DEVICE_CHECK
    assert all(s == ei.EI_OK for s in info["statuses"]), info["statuses"]
    # the regular build (this process): no checks, identical results
    assert not ei.ei_device_checks_enabled()
    assert ei.ei_selftest_device_check() == 0
    ref, statuses = _evaluations()
    assert all(s == ei.EI_OK for s in statuses)
    got = info["results"]
    assert sorted(got) == sorted(ref)
    for k, (S, g) in ref.items():
        assert got[k][0] == S, (k, got[k][0], S)          # objectives equal bit for bit
        assert got[k][1] == g, k                          # gradients / iterates: equal bytes
