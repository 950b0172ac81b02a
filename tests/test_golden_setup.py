"""The constants the paper prints for its acquisition and reconstruction
(fixture tests/golden/paper_setup.txt, each value with its section) are the
ones the synthetic inputs, the model and the resolution study use."""
import inspect
import os

import pytest

from paper_2202_08627_gb300 import inputs, metrics, ring_study

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_setup.txt")


def _paper():
    vals = {}
    for line in open(GOLDEN):
        body = line.split("#", 1)[0].strip()
        if body:
            k, v = (x.strip() for x in body.split("=", 1))
            vals[k] = float(v)
    return vals


def test_fixture_is_complete():
    assert set(_paper()) == {"z_cm", "detector_mask_pitch_cm", "sample_mask_pitch_cm",
                             "flat_scan_steps", "flat_scan_repeats", "projections",
                             "slice_voxels", "lambda", "gamma", "frc_half_projections",
                             "frc_crop_voxels", "frc_cutoff"}


def test_model_constants_are_the_papers():
    p = _paper()
    assert inputs.Z_CM == p["z_cm"]
    assert inputs.PERIOD_CM == pytest.approx(p["detector_mask_pitch_cm"], rel=1e-12)
    assert inputs.LAMBDA == p["lambda"]
    # the shift per unit dR[delta]/dt is z / period: 20 cm / 48 um
    assert inputs.Z_CM / inputs.PERIOD_CM == pytest.approx(20.0 / 0.0048, rel=1e-12)


def test_resolution_study_follows_the_papers_protocol():
    p = _paper()
    assert ring_study.FLAT_STEPS == p["flat_scan_steps"]
    assert ring_study.flat_positions()[-1] - ring_study.flat_positions()[0] == pytest.approx(1.0)
    assert inspect.signature(metrics.frc_resolution).parameters["cutoff"].default == p["frc_cutoff"]
    # the FRC crop: the central 140 of 220 voxels, as a fraction of the slice
    assert ring_study.FRC_CROP == p["frc_crop_voxels"] / p["slice_voxels"]
    # odd / even halves of the paper's 400 projections
    assert 2 * p["frc_half_projections"] == p["projections"]
