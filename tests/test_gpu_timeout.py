"""Failure detection on the GPU without a fault: the bounded mbarrier wait the
bulk-copy kernels use gives up on a barrier that nothing completes, records
EI_ERR_TIMEOUT, and the context keeps working."""
import numpy as np
import pytest

import oracle
from paper_2202_08627_gb300 import inputs
from tests.problems import gpu_geometry, oracle_geometry, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    import time
    from paper_2202_08627_gb300 import ei
    t0 = time.perf_counter()
    assert ei.ei_selftest_wait_timeout(20000) == ei.EI_ERR_TIMEOUT      # 20 ms limit
    assert time.perf_counter() - t0 < 10.0
    # the same context computes correctly afterwards
    spec = inputs.make_slice(3, 37, 23, 61, 3)
    geom = oracle_geometry(spec)
    G = gpu_geometry([spec], [geom])
    proj = G.empty("proj")
    ei.ei_project(G, G.pack_volume([spec.truth]), proj)
    got = G.unpack_proj(proj)[0]
    for c in range(3):
        assert rel_l2(got[c], oracle.project(spec.truth[c], geom)) <= 1e-5
    # and a second self-test reports the same
    assert ei.ei_selftest_wait_timeout(1000) == ei.EI_ERR_TIMEOUT
