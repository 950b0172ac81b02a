"""The C-ABI library loads and exports every entry point include/ei.h
declares; host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2202_08627_gb300 import build, ei
    build.build()
    return ei.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ei.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ei_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ei_setup_geometry", "ei_forward", "ei_objective_grad", "ei_reconstruct",
                     "ei_destroy_geometry", "ei_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2202_08627_gb300 import ei
    assert sorted(ei.EXPORTED) == declared_functions()


def test_status_strings(lib):
    from paper_2202_08627_gb300 import ei
    for code in range(8):
        assert ei.ei_status_string(code).startswith("EI_")
    assert "unknown" in ei.ei_status_string(99)


def test_default_options(lib):
    from paper_2202_08627_gb300 import ei
    o = ei.ei_default_solve_opts()
    assert (o.tol, o.max_iter, o.lbfgs_m, o.c1, o.max_trials) == (1e-6, 100, 10, 1e-4, 20)
    assert (o.use_graph, o.resume, o.max_seconds) == (1, 0, 0.0)
    assert ctypes.sizeof(ei.ei_solve_opts) == 56      # the C layout (gcc: 56 B, max_seconds at 48)
    assert ei.ei_solve_opts.max_seconds.offset == 48


def test_checkpoint_calls_reject_bad_arguments_before_touching_the_gpu(lib):
    from paper_2202_08627_gb300 import ei
    n = ctypes.c_size_t(0)
    buf = (ctypes.c_char * 16)()
    assert lib.ei_solver_state_size(None, 10, ctypes.byref(n)) == ei.EI_ERR_ARG
    assert lib.ei_solver_save(None, buf, 16) == ei.EI_ERR_ARG
    assert lib.ei_solver_load(None, 10, buf, 16) == ei.EI_ERR_ARG


def test_setup_rejects_bad_arguments_before_touching_the_gpu(lib):
    from paper_2202_08627_gb300 import ei
    flat = np.ones(8, np.float32)
    good = dict(n_m=3, m=[-0.5, 0, 0.5], z_cm=20.0, period_cm=48e-4, kappa_sigma=0.1,
                flat_A=flat, flat_c=flat * 0, flat_w=flat * 0.25, n=8, n_theta=4, n_det=8,
                pitch_cm=0.01)
    bad_cases = [dict(n_m=0), dict(n_m=40, m=np.zeros(40)), dict(period_cm=0.0), dict(n=0),
                 dict(n_det=ei.EI_MAX_NDET + 1), dict(pitch_cm=-1.0), dict(scale=(1, 0, 1)),
                 dict(lam=(1, -1, 1)), dict(n_slices=0)]
    for bad in bad_cases:
        with pytest.raises(ei.EIError) as err:
            ei.ei_setup_geometry(**{**good, **bad})
        assert err.value.status == ei.EI_ERR_ARG, bad


def test_wait_selftest_rejects_bad_arguments_before_touching_the_gpu(lib):
    from paper_2202_08627_gb300 import ei
    st = ctypes.c_int(-1)
    assert lib.ei_selftest_wait_timeout(0, ctypes.byref(st)) == ei.EI_ERR_ARG
    assert lib.ei_selftest_wait_timeout(2000001, ctypes.byref(st)) == ei.EI_ERR_ARG
    assert lib.ei_selftest_wait_timeout(1000, None) == ei.EI_ERR_ARG
    assert st.value == -1


def test_null_handle_calls_are_argument_errors(lib):
    from paper_2202_08627_gb300 import ei
    assert lib.ei_project(None, None, None, None) == ei.EI_ERR_ARG
    assert lib.ei_objective_grad(None, None, None, None, None, None) == ei.EI_ERR_ARG
    assert lib.ei_reconstruct(None, None, None, None, None, None) == ei.EI_ERR_ARG
    lib.ei_destroy_geometry(None)


def test_allocation_failure_trigger_without_a_gpu(lib):
    """The trigger is host state: arming, reading and disarming it need no
    device; nothing is allocated while no geometry exists."""
    from paper_2202_08627_gb300 import ei
    assert lib.ei_fail_alloc_after(-2) == ei.EI_ERR_ARG
    assert lib.ei_fail_alloc_pending(None) == ei.EI_ERR_ARG
    assert lib.ei_live_allocations(None) == ei.EI_ERR_ARG
    ei.ei_fail_alloc_after(3)
    assert ei.ei_fail_alloc_pending() == 3
    ei.ei_fail_alloc_after(-1)
    assert ei.ei_fail_alloc_pending() == -1
    assert ei.ei_live_allocations() == 0


def test_solve_report_layout_and_ring_modes_argument_checks(lib):
    from paper_2202_08627_gb300 import ei
    # six pointers, int + padding, double, then the per-slice projection and
    # adjoint counts (the C layout on both the x86 and the Arm build)
    assert ctypes.sizeof(ei.ei_solve_report) == 80
    assert ei.ei_solve_report.seconds.offset == 56
    assert ei.ei_solve_report.slice_projections.offset == 64
    assert ei.ei_solve_report.slice_adjoints.offset == 72
    assert lib.ei_set_ring_modes(None, 4) == ei.EI_ERR_ARG


def test_regular_build_has_no_device_checks(lib):
    assert lib.ei_device_checks_enabled() == 0
