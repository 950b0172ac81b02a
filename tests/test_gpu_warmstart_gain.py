"""What the learned warm start gains over the method without it.

A small U-Net (3 levels, 32 base channels) is trained on the GPU by the
library's own kernels on (single-shot, converged) pairs that the plain method
generates for 512 synthetic 64x64 slices (90 angles, 96 pixels, M = 7); on 64
held-out slices (other seeds) the plain L-BFGS is then run to the same
relative-change tolerance from x0 = 0, from the single-shot reconstruction and
from the network's output.  The learned start needs clearly fewer iterations
than both, and the solves reach the same objective (the tolerance, not the
start, decides the final accuracy)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


def test_learned_start_saves_iterations():
    from paper_2202_08627_gb300 import warmstart
    shape = (64, 90, 96)
    pairs, it = warmstart.generate_pairs([shape] * 512, 1_000_000, 7)
    assert np.all(it > 0)
    net = warmstart.WarmStartNet(levels=3, base=32, crop=64, batch=16, seed=0)
    hist = warmstart.train(net, pairs, 15, 1e-3, lr_final=5e-5, steps_per_epoch=64)
    assert hist[-1] < 0.2 * hist[0]
    ev = warmstart.evaluate(net, [shape] * 64, 2_000_000, 7)
    zero, ss, cnn = ev["zero"], ev["single_shot"], ev["cnn"]
    assert zero["converged"] == ss["converged"] == cnn["converged"] == 64
    assert cnn["iterations_mean"] <= 0.85 * zero["iterations_mean"], ev
    assert cnn["iterations_mean"] < ss["iterations_mean"], ev
    assert cnn["f_final_rel_diff_vs_zero_max"] <= 1e-3
    net.close()
