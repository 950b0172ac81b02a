"""The synthetic workloads are the recipe they state: sizes, the spread of
detector widths, the bytes they occupy, and determinism (no GPU needed)."""
import numpy as np

from paper_2202_08627_gb300 import workloads


def test_uneven_batch_recipe():
    wl = workloads.uneven1024()
    assert wl.n_slices == 256 and wl.n_m == 7
    assert [n for n, _, _ in wl.slices] == [1024, 512] * 128       # interleaved halves
    assert {nth for _, nth, _ in wl.slices} == {1800}
    dets = np.array([nd for _, _, nd in wl.slices])
    assert set(dets) == {1024, 1152, 1280, 1408, 1536}               # every width drawn
    assert abs(dets.mean() - 1280) < 40                              # uniform over the five
    assert wl.voxel_equiv_1024() == 160.0                            # 128 + 128 / 4
    assert 16.0e9 < wl.meas_bytes() < 17.0e9                         # "about 16.5 GB"
    assert workloads.uneven1024().slices == wl.slices                # seeded


def test_sub_batches_and_profile_case():
    wl = workloads.uneven1024()
    pure = workloads.pure1024()
    assert pure.slices == [s for s in wl.slices if s[0] == 1024] and pure.n_slices == 128
    b8 = workloads.batch8x1024()
    assert b8.slices == [(1024, 1800, 1536)] * 8
    assert abs(16 * 1024 ** 2 * 8 - 134e6) < 1e6                     # the packed volume
    assert abs(b8.meas_bytes() - 620e6) < 2e6                        # measured ICs > L2 (129 MB)


def test_algorithmic_bytes_per_evaluation():
    """Projector + adjoint: 48 n^2 + 28 n_theta n_det per slice (the
    headline metric's numerator); IC: (28 + 4 M) n_theta n_det."""
    for wl in (workloads.small(), workloads.check128(), workloads.uneven1024()):
        fa = sum(48 * n * n + 28 * nth * nd for n, nth, nd in wl.slices)
        assert wl.fwd_bytes() + wl.adj_bytes() == fa
        assert wl.ic_bytes() == sum((28 + 4 * wl.n_m) * nth * nd for _, nth, nd in wl.slices)
        assert wl.taps() == sum(2 * n * n * nth for n, nth, _ in wl.slices)


def test_every_named_workload_builds():
    for name, make in workloads.WORKLOADS.items():
        wl = make()
        assert wl.name == name and wl.n_slices >= 1
        assert all(n >= 1 and nth >= 1 and nd >= 1 for n, nth, nd in wl.slices)
