"""Thin Python binding of libei.so (C ABI in include/ei.h).

Argument marshalling only: every step of the reconstruction runs in the CUDA
kernels behind the ABI.  Functions keep the ABI's names.  Arrays are PyTorch
CUDA tensors (float32, contiguous, 16-byte aligned) in the layouts documented
in include/ei.h; ``pack_volume`` / ``unpack_volume`` and friends convert
between those layouts and per-slice arrays.

The library is loaded on first use.  If it has not been built (see
``paper_2202_08627_gb300.build``) the import of the library raises — there is
no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libei.so")

EI_OK, EI_ERR_ARG, EI_ERR_CUDA, EI_ERR_NONFINITE, EI_ERR_LINESEARCH = 0, 1, 2, 3, 4
EI_ERR_TIMEOUT, EI_ERR_DEVICE_CHECK, EI_ERR_ALLOC = 5, 6, 7
EI_MAX_NDET = 8192
EI_MAX_NM = 32

c_int, c_double, c_void_p, c_int64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64


class ei_slice_dims(ctypes.Structure):
    _fields_ = [("n", c_int), ("n_theta", c_int), ("n_det", c_int), ("pitch_cm", c_double)]


class ei_geometry_desc(ctypes.Structure):
    _fields_ = [("n", c_int), ("n_theta", c_int), ("n_det", c_int), ("n_m", c_int),
                ("pitch_cm", c_double),
                ("theta", ctypes.POINTER(c_double)), ("m", ctypes.POINTER(c_double)),
                ("z_cm", c_double), ("period_cm", c_double), ("kappa_sigma", c_double),
                ("flat_A", c_void_p), ("flat_c", c_void_p), ("flat_w", c_void_p),
                ("lambda_", c_double * 3), ("scale", c_double * 3),
                ("m_o", c_void_p), ("m_r", c_void_p)]


class ei_slice_layout(ctypes.Structure):
    _fields_ = [("n", c_int), ("n_theta", c_int), ("n_det", c_int), ("n_dp", c_int),
                ("n_m", c_int), ("pitch_cm", c_double),
                ("vol_offset", c_int64), ("vol_count", c_int64),
                ("proj_offset", c_int64), ("proj_count", c_int64),
                ("sino4_offset", c_int64), ("sino4_count", c_int64),
                ("meas_offset", c_int64), ("meas_count", c_int64)]


class ei_layout(ctypes.Structure):
    _fields_ = [("n_slices", c_int), ("n_m", c_int),
                ("vol_count", c_int64), ("proj_count", c_int64), ("sino4_count", c_int64),
                ("meas_count", c_int64), ("workspace_bytes", c_int64)]


class ei_solve_opts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("max_iter", c_int), ("lbfgs_m", c_int), ("c1", c_double),
                ("max_trials", c_int), ("curv_eps", c_double), ("use_graph", c_int),
                ("resume", c_int), ("max_seconds", c_double)]


class ei_solve_report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.POINTER(c_int)), ("status", ctypes.POINTER(c_int)),
                ("converged", ctypes.POINTER(c_int)), ("f_final", ctypes.POINTER(c_double)),
                ("f_initial", ctypes.POINTER(c_double)),
                ("slice_evaluations", ctypes.POINTER(c_int)), ("evaluations", c_int),
                ("seconds", c_double), ("slice_projections", ctypes.POINTER(c_int)),
                ("slice_adjoints", ctypes.POINTER(c_int))]


class ei_peaks(ctypes.Structure):
    _fields_ = [("fp32_tflops", c_double), ("l1_load_tbs", c_double),
                ("smem_load_tbs", c_double), ("num_sms", c_int)]


class ei_profile(ctypes.Structure):
    _fields_ = [("launches", c_int64), ("project_launches", c_int64), ("ic_launches", c_int64),
                ("backproject_launches", c_int64), ("project_ms", c_double), ("ic_ms", c_double),
                ("backproject_ms", c_double)]


EXPORTED = ["ei_setup_geometry", "ei_destroy_geometry", "ei_get_layout", "ei_get_slice_layout",
            "ei_project", "ei_backproject", "ei_ic_model", "ei_forward", "ei_objective_grad",
            "ei_reconstruct", "ei_default_solve_opts", "ei_status_string", "ei_profile_enable",
            "ei_profile_read", "ei_objective_grad_noalloc", "ei_autotune", "ei_set_variant",
            "ei_get_variant", "ei_last_error", "ei_single_shot_fbp", "ei_unet_create",
            "ei_unet_destroy", "ei_unet_forward", "ei_unet_train_step", "ei_unet_num_params",
            "ei_unet_get_params", "ei_unet_set_params", "ei_unet_get_grads", "ei_set_ic_variant",
            "ei_get_ic_variant", "ei_measure_peaks", "ei_set_linked", "ei_offset_grad",
            "ei_set_offset_unknowns", "ei_get_offsets", "ei_single_shot_eq3",
            "ei_unet_set_tensor_path", "ei_set_flat_table", "ei_selftest_wait_timeout",
            "ei_solver_state_size", "ei_solver_save", "ei_solver_load",
            "ei_unet_get_optimizer", "ei_unet_set_optimizer", "ei_fail_alloc_after",
            "ei_fail_alloc_pending", "ei_live_allocations", "ei_set_ring_modes",
            "ei_device_checks_enabled", "ei_selftest_device_check"]
EI_OFFSET_MO, EI_OFFSET_MR = 1, 2
EI_TUNE_FORCE, EI_TUNE_NO_CACHE_WRITE = 1, 2
N_FWD_VARIANTS, N_ADJ_VARIANTS = 14, 14

_lib = None


def load_library(path: str = None) -> ctypes.CDLL:
    """Load libei.so (or the build at `path`, once, before any other call);
    raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("EI_LIBRARY", LIB_PATH)
    if not os.path.exists(path):
        raise RuntimeError("libei.so not found at %s: build it with "
                           "paper_2202_08627_gb300.build.build() (there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    lib.ei_setup_geometry.argtypes = [P(ei_geometry_desc), c_int, P(ei_slice_dims), P(c_void_p)]
    lib.ei_setup_geometry.restype = c_int
    lib.ei_destroy_geometry.argtypes = [c_void_p]
    lib.ei_destroy_geometry.restype = None
    lib.ei_get_layout.argtypes = [c_void_p, P(ei_layout)]
    lib.ei_get_layout.restype = c_int
    lib.ei_get_slice_layout.argtypes = [c_void_p, c_int, P(ei_slice_layout)]
    lib.ei_get_slice_layout.restype = c_int
    for name in ("ei_project", "ei_backproject", "ei_ic_model", "ei_forward", "ei_single_shot_fbp"):
        fn = getattr(lib, name)
        fn.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
        fn.restype = c_int
    lib.ei_objective_grad.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.ei_objective_grad.restype = c_int
    lib.ei_reconstruct.argtypes = [c_void_p, c_void_p, c_void_p, P(ei_solve_opts),
                                   P(ei_solve_report), c_void_p]
    lib.ei_reconstruct.restype = c_int
    lib.ei_default_solve_opts.argtypes = [P(ei_solve_opts)]
    lib.ei_default_solve_opts.restype = None
    lib.ei_profile_enable.argtypes = [c_void_p, c_int]
    lib.ei_profile_enable.restype = c_int
    lib.ei_profile_read.argtypes = [c_void_p, P(ei_profile)]
    lib.ei_profile_read.restype = c_int
    lib.ei_objective_grad_noalloc.argtypes = [P(ei_geometry_desc), c_void_p, c_void_p, c_void_p,
                                              c_void_p, c_void_p]
    lib.ei_objective_grad_noalloc.restype = c_int
    lib.ei_autotune.argtypes = [c_void_p, c_int, c_void_p]
    lib.ei_autotune.restype = c_int
    lib.ei_set_variant.argtypes = [c_void_p, c_int, c_int, c_int]
    lib.ei_set_variant.restype = c_int
    lib.ei_get_variant.argtypes = [c_void_p, P(c_int), P(c_int), P(c_int)]
    lib.ei_get_variant.restype = c_int
    lib.ei_unet_set_tensor_path.argtypes = [c_void_p, c_int]
    lib.ei_unet_set_tensor_path.restype = c_int
    lib.ei_single_shot_eq3.argtypes = [c_void_p, c_void_p, c_int, c_double, c_void_p, c_void_p]
    lib.ei_single_shot_eq3.restype = c_int
    lib.ei_set_offset_unknowns.argtypes = [c_void_p, c_int, c_double]
    lib.ei_set_offset_unknowns.restype = c_int
    lib.ei_set_ring_modes.argtypes = [c_void_p, c_int]
    lib.ei_set_ring_modes.restype = c_int
    lib.ei_get_offsets.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.ei_get_offsets.restype = c_int
    lib.ei_unet_get_optimizer.argtypes = [c_void_p, c_void_p, c_void_p, P(c_int)]
    lib.ei_unet_get_optimizer.restype = c_int
    lib.ei_unet_set_optimizer.argtypes = [c_void_p, c_void_p, c_void_p, c_int]
    lib.ei_unet_set_optimizer.restype = c_int
    lib.ei_solver_state_size.argtypes = [c_void_p, c_int, P(ctypes.c_size_t)]
    lib.ei_solver_state_size.restype = c_int
    lib.ei_solver_save.argtypes = [c_void_p, c_void_p, ctypes.c_size_t]
    lib.ei_solver_save.restype = c_int
    lib.ei_solver_load.argtypes = [c_void_p, c_int, c_void_p, ctypes.c_size_t]
    lib.ei_solver_load.restype = c_int
    lib.ei_selftest_wait_timeout.argtypes = [ctypes.c_uint, P(c_int)]
    lib.ei_selftest_wait_timeout.restype = c_int
    lib.ei_device_checks_enabled.argtypes = []
    lib.ei_device_checks_enabled.restype = c_int
    lib.ei_selftest_device_check.argtypes = [P(c_int)]
    lib.ei_selftest_device_check.restype = c_int
    lib.ei_fail_alloc_after.argtypes = [c_int]
    lib.ei_fail_alloc_after.restype = c_int
    lib.ei_fail_alloc_pending.argtypes = [P(c_int)]
    lib.ei_fail_alloc_pending.restype = c_int
    lib.ei_live_allocations.argtypes = [P(c_int64)]
    lib.ei_live_allocations.restype = c_int
    lib.ei_set_flat_table.argtypes = [c_void_p, c_void_p, c_int]
    lib.ei_set_flat_table.restype = c_int
    lib.ei_set_linked.argtypes = [c_void_p, c_double]
    lib.ei_set_linked.restype = c_int
    lib.ei_offset_grad.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.ei_offset_grad.restype = c_int
    lib.ei_measure_peaks.argtypes = [P(ei_peaks), c_void_p]
    lib.ei_measure_peaks.restype = c_int
    lib.ei_set_ic_variant.argtypes = [c_void_p, c_int]
    lib.ei_set_ic_variant.restype = c_int
    lib.ei_get_ic_variant.argtypes = [c_void_p, P(c_int)]
    lib.ei_get_ic_variant.restype = c_int
    lib.ei_unet_create.argtypes = [c_int, c_int, c_int, c_int, c_int, ctypes.c_ulonglong,
                                   P(c_void_p)]
    lib.ei_unet_create.restype = c_int
    lib.ei_unet_destroy.argtypes = [c_void_p]
    lib.ei_unet_destroy.restype = None
    lib.ei_unet_forward.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_void_p]
    lib.ei_unet_forward.restype = c_int
    lib.ei_unet_train_step.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_double,
                                       P(c_double), c_void_p]
    lib.ei_unet_train_step.restype = c_int
    lib.ei_unet_num_params.argtypes = [c_void_p]
    lib.ei_unet_num_params.restype = c_int64
    for name in ("ei_unet_get_params", "ei_unet_set_params", "ei_unet_get_grads"):
        getattr(lib, name).argtypes = [c_void_p, c_void_p]
        getattr(lib, name).restype = c_int
    lib.ei_last_error.argtypes = []
    lib.ei_last_error.restype = ctypes.c_char_p
    lib.ei_status_string.argtypes = [c_int]
    lib.ei_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


class EIError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        lib = load_library()
        msg = lib.ei_status_string(status).decode()
        if status in (EI_ERR_CUDA, EI_ERR_ALLOC):
            msg += " (%s)" % lib.ei_last_error().decode()
        super().__init__("%s failed: %s" % (where, msg))


def _check(status: int, where: str):
    if status != EI_OK:
        raise EIError(status, where)


def ei_status_string(status: int) -> str:
    return load_library().ei_status_string(status).decode()


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dptr(t, name: str, dtype=None) -> int:
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return int(t.data_ptr())


@dataclass
class SliceLayout:
    n: int
    n_theta: int
    n_det: int
    n_dp: int
    n_m: int
    pitch_cm: float
    vol_offset: int
    vol_count: int
    proj_offset: int
    proj_count: int
    sino4_offset: int
    sino4_count: int
    meas_offset: int
    meas_count: int


class Geometry:
    """Owns an ei_geometry handle (device workspace on the current device)."""

    def __init__(self, handle: int):
        self.handle = handle
        lib = load_library()
        lay = ei_layout()
        _check(lib.ei_get_layout(handle, ctypes.byref(lay)), "ei_get_layout")
        self.n_slices = lay.n_slices
        self.n_m = lay.n_m
        self.vol_count = lay.vol_count
        self.proj_count = lay.proj_count
        self.sino4_count = lay.sino4_count
        self.meas_count = lay.meas_count
        self.workspace_bytes = lay.workspace_bytes
        self.slices: List[SliceLayout] = []
        for s in range(self.n_slices):
            sl = ei_slice_layout()
            _check(lib.ei_get_slice_layout(handle, s, ctypes.byref(sl)), "ei_get_slice_layout")
            self.slices.append(SliceLayout(*[getattr(sl, f) for f, _ in sl._fields_]))

    def close(self):
        if self.handle:
            load_library().ei_destroy_geometry(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- layout marshalling (no arithmetic of the method)
    def empty(self, what: str, device="cuda"):
        import torch
        if what == "vol":
            return torch.zeros((self.vol_count, 4), dtype=torch.float32, device=device)
        if what == "proj":
            return torch.zeros(self.proj_count, dtype=torch.float32, device=device)
        if what == "sino4":
            return torch.zeros((self.sino4_count, 4), dtype=torch.float32, device=device)
        if what == "meas":
            return torch.zeros(self.meas_count, dtype=torch.float32, device=device)
        raise ValueError(what)

    def pack_volume(self, vols: Sequence[np.ndarray], device="cuda"):
        """[3][n][n] arrays per slice -> vol layout tensor [vol_count][4]."""
        import torch
        out = np.zeros((self.vol_count, 4), dtype=np.float32)
        for s, sl in enumerate(self.slices):
            v = np.asarray(vols[s], dtype=np.float32).reshape(3, sl.n * sl.n)
            out[sl.vol_offset:sl.vol_offset + sl.vol_count, :3] = v.T
        return torch.from_numpy(out).to(device)

    def unpack_volume(self, t) -> List[np.ndarray]:
        a = t.detach().cpu().numpy().reshape(self.vol_count, 4)
        return [a[sl.vol_offset:sl.vol_offset + sl.vol_count, :3].T.reshape(3, sl.n, sl.n).copy()
                for sl in self.slices]

    def pack_meas(self, meas: Sequence[np.ndarray], device="cuda"):
        """[M][n_theta][n_det] arrays per slice -> measurement layout tensor."""
        import torch
        out = np.zeros(self.meas_count, dtype=np.float32)
        for s, sl in enumerate(self.slices):
            blk = np.zeros((sl.n_m, sl.n_theta, sl.n_dp), dtype=np.float32)
            blk[:, :, :sl.n_det] = meas[s]
            out[sl.meas_offset:sl.meas_offset + sl.meas_count] = blk.ravel()
        return torch.from_numpy(out).to(device)

    def unpack_meas(self, t) -> List[np.ndarray]:
        a = t.detach().cpu().numpy()
        return [a[sl.meas_offset:sl.meas_offset + sl.meas_count]
                .reshape(sl.n_m, sl.n_theta, sl.n_dp)[:, :, :sl.n_det].copy() for sl in self.slices]

    def pack_proj(self, projs: Sequence[np.ndarray], device="cuda"):
        import torch
        out = np.zeros(self.proj_count, dtype=np.float32)
        for s, sl in enumerate(self.slices):
            blk = np.zeros((3, sl.n_theta, sl.n_dp), dtype=np.float32)
            blk[:, :, :sl.n_det] = projs[s]
            out[sl.proj_offset:sl.proj_offset + sl.proj_count] = blk.ravel()
        return torch.from_numpy(out).to(device)

    def unpack_proj(self, t) -> List[np.ndarray]:
        a = t.detach().cpu().numpy()
        return [a[sl.proj_offset:sl.proj_offset + sl.proj_count]
                .reshape(3, sl.n_theta, sl.n_dp)[:, :, :sl.n_det].copy() for sl in self.slices]

    def pack_sino4(self, sinos: Sequence[np.ndarray], device="cuda"):
        """[3][n_theta][n_det] arrays per slice -> sino4 layout tensor [sino4_count][4]."""
        import torch
        out = np.zeros((self.sino4_count, 4), dtype=np.float32)
        for s, sl in enumerate(self.slices):
            blk = np.zeros((sl.n_theta, sl.n_dp, 3), dtype=np.float32)
            blk[:, :sl.n_det, :] = np.moveaxis(np.asarray(sinos[s]), 0, -1)
            out[sl.sino4_offset:sl.sino4_offset + sl.sino4_count, :3] = blk.reshape(-1, 3)
        return torch.from_numpy(out).to(device)


def ei_setup_geometry(n_m: int, m: Sequence[float], z_cm: float, period_cm: float,
                      kappa_sigma: float, flat_A, flat_c, flat_w, lam=(1e-2, 1e-2, 1e-2),
                      scale=(1.0, 1e-6, 1.0), n: int = 0, n_theta: int = 0, n_det: int = 0,
                      pitch_cm: float = 0.0, n_slices: int = 1,
                      per_slice: Optional[Sequence[tuple]] = None, theta=None, m_o=None,
                      m_r=None) -> Geometry:
    """Create a geometry.  flat_* / m_o / m_r: numpy arrays (host) or CUDA
    tensors; per_slice: list of (n, n_theta, n_det, pitch_cm) for uneven
    batches (then n_slices = len(per_slice))."""
    lib = load_library()
    keep = []

    def fptr(a):
        if a is None:
            return None
        try:
            import torch
            if isinstance(a, torch.Tensor):
                a = a.contiguous().float()
                keep.append(a)
                return a.data_ptr()
        except ImportError:
            pass
        arr = np.ascontiguousarray(a, dtype=np.float32)
        keep.append(arr)
        return arr.ctypes.data

    d = ei_geometry_desc()
    d.n, d.n_theta, d.n_det, d.n_m = int(n), int(n_theta), int(n_det), int(n_m)
    d.pitch_cm = float(pitch_cm)
    m_arr = np.ascontiguousarray(m, dtype=np.float64)
    keep.append(m_arr)
    d.m = m_arr.ctypes.data_as(ctypes.POINTER(c_double))
    if theta is not None:
        th = np.ascontiguousarray(theta, dtype=np.float64)
        keep.append(th)
        d.theta = th.ctypes.data_as(ctypes.POINTER(c_double))
    d.z_cm, d.period_cm, d.kappa_sigma = float(z_cm), float(period_cm), float(kappa_sigma)
    d.flat_A, d.flat_c, d.flat_w = fptr(flat_A), fptr(flat_c), fptr(flat_w)
    d.lambda_[:] = [float(v) for v in lam]
    d.scale[:] = [float(v) for v in scale]
    d.m_o, d.m_r = fptr(m_o), fptr(m_r)
    ps = None
    if per_slice is not None:
        n_slices = len(per_slice)
        ps = (ei_slice_dims * n_slices)(*[ei_slice_dims(int(a), int(b), int(c), float(e))
                                          for (a, b, c, e) in per_slice])
    h = c_void_p()
    _check(lib.ei_setup_geometry(ctypes.byref(d), int(n_slices), ps, ctypes.byref(h)),
           "ei_setup_geometry")
    return Geometry(h.value)


def ei_destroy_geometry(geom: Geometry) -> None:
    geom.close()


def _check_size(t, count: int, name: str):
    if t.numel() < count:
        raise ValueError("%s holds %d floats, the layout needs %d" % (name, t.numel(), count))
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)


def ei_project(geom: Geometry, vol, proj, stream=None) -> None:
    import torch
    _check_size(vol, 4 * geom.vol_count, "vol")
    _check_size(proj, geom.proj_count, "proj")
    _check(load_library().ei_project(geom.handle, _dptr(vol, "vol", torch.float32),
                                     _dptr(proj, "proj", torch.float32), _stream_ptr(stream)),
           "ei_project")


def ei_backproject(geom: Geometry, sino4, vol, stream=None) -> None:
    import torch
    _check_size(sino4, 4 * geom.sino4_count, "sino4")
    _check_size(vol, 4 * geom.vol_count, "vol")
    _check(load_library().ei_backproject(geom.handle, _dptr(sino4, "sino4", torch.float32),
                                         _dptr(vol, "vol", torch.float32), _stream_ptr(stream)),
           "ei_backproject")


def ei_ic_model(geom: Geometry, proj, s_mod, stream=None) -> None:
    import torch
    _check_size(proj, geom.proj_count, "proj")
    _check_size(s_mod, geom.meas_count, "s_mod")
    _check(load_library().ei_ic_model(geom.handle, _dptr(proj, "proj", torch.float32),
                                      _dptr(s_mod, "s_mod", torch.float32), _stream_ptr(stream)),
           "ei_ic_model")


def ei_forward(geom: Geometry, vol, s_mod, stream=None) -> None:
    import torch
    _check_size(vol, 4 * geom.vol_count, "vol")
    _check_size(s_mod, geom.meas_count, "s_mod")
    _check(load_library().ei_forward(geom.handle, _dptr(vol, "vol", torch.float32),
                                     _dptr(s_mod, "s_mod", torch.float32), _stream_ptr(stream)),
           "ei_forward")


def ei_single_shot_fbp(geom: Geometry, s_exp, vol_out, stream=None) -> None:
    """Non-iterative reconstruction (moment retrieval + filtered back-projection)."""
    import torch
    _check_size(s_exp, geom.meas_count, "s_exp")
    _check_size(vol_out, 4 * geom.vol_count, "vol_out")
    _check(load_library().ei_single_shot_fbp(geom.handle, _dptr(s_exp, "s_exp", torch.float32),
                                             _dptr(vol_out, "vol_out", torch.float32),
                                             _stream_ptr(stream)), "ei_single_shot_fbp")


def ei_objective_grad(geom: Geometry, vol, s_exp, S_out, grad=None, stream=None) -> None:
    """S_out: float64 tensor [n_slices] (CUDA or CPU); grad: vol-layout tensor or None."""
    import torch
    _check_size(vol, 4 * geom.vol_count, "vol")
    _check_size(s_exp, geom.meas_count, "s_exp")
    if S_out.dtype != torch.float64 or S_out.numel() < geom.n_slices:
        raise ValueError("S_out must be a float64 tensor of n_slices entries")
    gp = None
    if grad is not None:
        _check_size(grad, 4 * geom.vol_count, "grad")
        gp = _dptr(grad, "grad", torch.float32)
    _check(load_library().ei_objective_grad(geom.handle, _dptr(vol, "vol", torch.float32),
                                            _dptr(s_exp, "s_exp", torch.float32),
                                            _dptr(S_out, "S_out"), gp, _stream_ptr(stream)),
           "ei_objective_grad")


def ei_default_solve_opts() -> ei_solve_opts:
    o = ei_solve_opts()
    load_library().ei_default_solve_opts(ctypes.byref(o))
    return o


@dataclass
class SolveReport:
    iterations: np.ndarray
    status: np.ndarray
    converged: np.ndarray
    f_final: np.ndarray
    f_initial: np.ndarray
    slice_evaluations: np.ndarray
    evaluations: int
    seconds: float
    return_status: int
    slice_projections: np.ndarray = None
    slice_adjoints: np.ndarray = None


def ei_reconstruct(geom: Geometry, s_exp, vol_inout, tol=1e-6, max_iter=100, lbfgs_m=10,
                   c1=1e-4, max_trials=20, curv_eps=1e-10, use_graph=True, stream=None,
                   raise_on_error: bool = True, resume: bool = False,
                   max_seconds: float = 0.0) -> SolveReport:
    """Batched L-BFGS minimisation of S.  s_exp / vol_inout: CUDA tensors, or
    pinned/pageable CPU tensors (the library stages host arrays).  resume:
    continue from the geometry's solver state (the last solve or
    ei_solver_load) instead of starting at vol_inout.  max_seconds > 0: time
    budget of the call; slices it stops report EI_ERR_TIMEOUT (not raised) and
    continue exactly under resume=True."""
    import torch
    if s_exp.numel() < geom.meas_count or vol_inout.numel() < 4 * geom.vol_count:
        raise ValueError("s_exp / vol_inout smaller than the layout")
    o = ei_solve_opts(float(tol), int(max_iter), int(lbfgs_m), float(c1), int(max_trials),
                      float(curv_eps), int(bool(use_graph)), int(bool(resume)),
                      float(max_seconds))
    S = geom.n_slices
    it = np.zeros(S, np.int32)
    st = np.zeros(S, np.int32)
    cv = np.zeros(S, np.int32)
    ff = np.zeros(S, np.float64)
    f0 = np.zeros(S, np.float64)
    ev = np.zeros(S, np.int32)
    npj = np.zeros(S, np.int32)
    nad = np.zeros(S, np.int32)
    ip = ctypes.POINTER(c_int)
    dp = ctypes.POINTER(c_double)
    rep = ei_solve_report(it.ctypes.data_as(ip), st.ctypes.data_as(ip), cv.ctypes.data_as(ip),
                          ff.ctypes.data_as(dp), f0.ctypes.data_as(dp), ev.ctypes.data_as(ip),
                          0, 0.0, npj.ctypes.data_as(ip), nad.ctypes.data_as(ip))
    rc = load_library().ei_reconstruct(geom.handle, _dptr(s_exp, "s_exp", torch.float32),
                                       _dptr(vol_inout, "vol_inout", torch.float32),
                                       ctypes.byref(o), ctypes.byref(rep), _stream_ptr(stream))
    out = SolveReport(it, st, cv, ff, f0, ev, rep.evaluations, rep.seconds, rc, npj, nad)
    budget_stop = rc == EI_ERR_TIMEOUT and max_seconds > 0 and bool((st == EI_ERR_TIMEOUT).any())
    if raise_on_error and rc not in (EI_OK, EI_ERR_LINESEARCH, EI_ERR_NONFINITE) and not budget_stop:
        raise EIError(rc, "ei_reconstruct")
    return out


def ei_solver_state_size(geom: Geometry, lbfgs_m: int = 10) -> int:
    n = ctypes.c_size_t(0)
    _check(load_library().ei_solver_state_size(geom.handle, int(lbfgs_m), ctypes.byref(n)),
           "ei_solver_state_size")
    return n.value


def ei_solver_save(geom: Geometry, lbfgs_m: int = 10) -> np.ndarray:
    """The solver state of the last solve as a host byte array."""
    buf = np.empty(ei_solver_state_size(geom, lbfgs_m), np.uint8)
    _check(load_library().ei_solver_save(geom.handle, buf.ctypes.data, buf.nbytes),
           "ei_solver_save")
    return buf


def ei_solver_load(geom: Geometry, buf: np.ndarray, lbfgs_m: int = 10) -> None:
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(load_library().ei_solver_load(geom.handle, int(lbfgs_m), buf.ctypes.data, buf.nbytes),
           "ei_solver_load")


def ei_profile_enable(geom: Geometry, on: bool = True) -> None:
    _check(load_library().ei_profile_enable(geom.handle, int(bool(on))), "ei_profile_enable")


def ei_profile_read(geom: Geometry) -> dict:
    p = ei_profile()
    _check(load_library().ei_profile_read(geom.handle, ctypes.byref(p)), "ei_profile_read")
    return {f: getattr(p, f) for f, _ in p._fields_}


def ei_objective_grad_noalloc(n: int, n_theta: int, n_det: int, pitch_cm: float, n_m: int,
                              m: Sequence[float], z_cm: float, period_cm: float,
                              kappa_sigma: float, flat_A, flat_c, flat_w, vol, s_exp, S_out,
                              grad=None, lam=(1e-2, 1e-2, 1e-2), scale=(1.0, 1e-6, 1.0),
                              theta=None, m_o=None, m_r=None, stream=None) -> None:
    """S and its gradient for one slice without any device allocation, for
    callers that may not allocate GPU memory (a framework that owns the device
    memory, or a loop that cannot afford cudaMalloc's synchronisation).
    Arguments as ei_setup_geometry (one uniform slice) plus ei_objective_grad's
    arrays; flat_* / m_o / m_r are numpy arrays or contiguous float32 CUDA
    tensors (other tensors are refused rather than converted, which would
    allocate)."""
    import torch
    keep = []

    def fptr(a):
        if a is None:
            return None
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float32 or not a.is_contiguous() or not a.is_cuda:
                raise ValueError("per-pixel tensors must be contiguous float32 CUDA tensors")
            return a.data_ptr()
        arr = np.ascontiguousarray(a, dtype=np.float32)
        keep.append(arr)
        return arr.ctypes.data

    d = ei_geometry_desc()
    d.n, d.n_theta, d.n_det, d.n_m = int(n), int(n_theta), int(n_det), int(n_m)
    d.pitch_cm = float(pitch_cm)
    m_arr = np.ascontiguousarray(m, dtype=np.float64)
    keep.append(m_arr)
    d.m = m_arr.ctypes.data_as(ctypes.POINTER(c_double))
    if theta is not None:
        th = np.ascontiguousarray(theta, dtype=np.float64)
        keep.append(th)
        d.theta = th.ctypes.data_as(ctypes.POINTER(c_double))
    d.z_cm, d.period_cm, d.kappa_sigma = float(z_cm), float(period_cm), float(kappa_sigma)
    d.flat_A, d.flat_c, d.flat_w = fptr(flat_A), fptr(flat_c), fptr(flat_w)
    d.lambda_[:] = [float(v) for v in lam]
    d.scale[:] = [float(v) for v in scale]
    d.m_o, d.m_r = fptr(m_o), fptr(m_r)
    if S_out.dtype != torch.float64 or S_out.numel() < 1:
        raise ValueError("S_out must be a float64 tensor")
    gp = None if grad is None else _dptr(grad, "grad", torch.float32)
    _check(load_library().ei_objective_grad_noalloc(
        ctypes.byref(d), _dptr(vol, "vol", torch.float32), _dptr(s_exp, "s_exp", torch.float32),
        _dptr(S_out, "S_out"), gp, _stream_ptr(stream)), "ei_objective_grad_noalloc")


def ei_autotune(geom: Geometry, force: bool = False, write_cache: bool = True, stream=None):
    """Time the projector/adjoint variants on this geometry, select the fastest
    (cached on disk); returns (fwd_variant, adj_variant, persistent)."""
    flags = (EI_TUNE_FORCE if force else 0) | (0 if write_cache else EI_TUNE_NO_CACHE_WRITE)
    _check(load_library().ei_autotune(geom.handle, flags, _stream_ptr(stream)), "ei_autotune")
    return ei_get_variant(geom)


LAUNCH_PER_ITEM, LAUNCH_PERSISTENT, LAUNCH_SM_CHUNKS = 0, 1, 2


def ei_set_variant(geom: Geometry, fwd_variant: int, adj_variant: int, persistent: int) -> None:
    """Projector and adjoint variants and their launch mode: 0 (or False) one
    block per work item, 1 (or True) a persistent grid with one work counter,
    2 a persistent grid whose blocks first take their SM's chunk of items."""
    _check(load_library().ei_set_variant(geom.handle, int(fwd_variant), int(adj_variant),
                                         int(persistent)), "ei_set_variant")


def ei_get_variant(geom: Geometry):
    f, a, p = c_int(), c_int(), c_int()
    _check(load_library().ei_get_variant(geom.handle, ctypes.byref(f), ctypes.byref(a),
                                         ctypes.byref(p)), "ei_get_variant")
    return f.value, a.value, p.value


def ei_single_shot_eq3(geom: Geometry, s_exp, m_index: int, gamma: float, vol_out, stream=None):
    """The paper's single-shot retrieval (Eq. 3) from one mask position and its
    FBP into vol_out: (h, gamma h, 0) per voxel."""
    _check_size(s_exp, geom.meas_count, "s_exp")
    _check_size(vol_out, geom.vol_count * 4, "vol_out")
    _check(load_library().ei_single_shot_eq3(geom.handle, _dptr(s_exp, "s_exp"), int(m_index),
                                             float(gamma), _dptr(vol_out, "vol_out"),
                                             _stream_ptr(stream)), "ei_single_shot_eq3")
    return vol_out


def ei_set_offset_unknowns(geom: Geometry, which: int, scale: float = 0.01) -> None:
    """Eq. 4's offsets among ei_reconstruct's unknowns: which = EI_OFFSET_MO |
    EI_OFFSET_MR (0 = fixed), solver scaling m / scale."""
    _check(load_library().ei_set_offset_unknowns(geom.handle, int(which), float(scale)),
           "ei_set_offset_unknowns")


def ei_set_ring_modes(geom: Geometry, K: int) -> None:
    """Restrict the solver's m_r steps to ring frequencies: orthogonal to the K
    lowest DCT-II modes across each slice's detector (0 = no restriction)."""
    _check(load_library().ei_set_ring_modes(geom.handle, int(K)), "ei_set_ring_modes")


def ei_get_offsets(geom: Geometry):
    """The geometry's current (m_o [sum n_theta], m_r [sum n_det]) as numpy arrays."""
    n_th = sum(sl.n_theta for sl in geom.slices)
    n_px = sum(sl.n_det for sl in geom.slices)
    m_o = np.zeros(n_th, np.float32)
    m_r = np.zeros(n_px, np.float32)
    _check(load_library().ei_get_offsets(geom.handle, m_o.ctypes.data, m_r.ctypes.data),
           "ei_get_offsets")
    return m_o, m_r


def ei_selftest_wait_timeout(limit_us: int) -> int:
    """Runs the bounded mbarrier wait on a barrier nothing completes, limited to
    limit_us; returns the status the kernel recorded (EI_ERR_TIMEOUT expected)."""
    st = c_int(-1)
    _check(load_library().ei_selftest_wait_timeout(int(limit_us), ctypes.byref(st)),
           "ei_selftest_wait_timeout")
    return st.value


def ei_device_checks_enabled() -> bool:
    """True for the build with device-side bounds checks (libei_check.so)."""
    return bool(load_library().ei_device_checks_enabled())


def ei_selftest_device_check() -> int:
    """Runs a checked read whose index leaves its logical range but not its
    buffer; returns the recorded status (EI_ERR_DEVICE_CHECK in the check
    build, 0 in the regular one)."""
    st = c_int(-1)
    _check(load_library().ei_selftest_device_check(ctypes.byref(st)), "ei_selftest_device_check")
    return st.value


def ei_fail_alloc_after(n: int) -> None:
    """Host-side failure injection: the next n device allocations of the
    library succeed and the one after them fails as out of memory (n = -1
    disarms)."""
    _check(load_library().ei_fail_alloc_after(int(n)), "ei_fail_alloc_after")


def ei_fail_alloc_pending() -> int:
    """Allocations still to pass before the armed failure, -1 when none is armed."""
    n = c_int(0)
    _check(load_library().ei_fail_alloc_pending(ctypes.byref(n)), "ei_fail_alloc_pending")
    return n.value


def ei_live_allocations() -> int:
    """Device allocations the library currently holds."""
    n = c_int64(0)
    _check(load_library().ei_live_allocations(ctypes.byref(n)), "ei_live_allocations")
    return n.value


def ei_set_flat_table(geom: Geometry, table) -> None:
    """Sampled flat IC [sum n_det][K] (f(t, k / K) over one mask period, float32
    numpy array or CUDA tensor); None restores the Gaussian flat."""
    lib = load_library()
    if table is None:
        _check(lib.ei_set_flat_table(geom.handle, None, 0), "ei_set_flat_table")
        return
    n_px = sum(sl.n_det for sl in geom.slices)
    if len(table.shape) != 2 or table.shape[0] != n_px:
        raise ValueError("flat table must be [%d][K], got %s" % (n_px, tuple(table.shape)))
    K = int(table.shape[1])
    if isinstance(table, np.ndarray):
        host = np.ascontiguousarray(table, dtype=np.float32)
        _check(lib.ei_set_flat_table(geom.handle, host.ctypes.data, K), "ei_set_flat_table")
    else:
        dev = table.contiguous().float()
        _check(lib.ei_set_flat_table(geom.handle, _dptr(dev, "table"), K), "ei_set_flat_table")


def ei_set_linked(geom: Geometry, gamma: float) -> None:
    """Linked single unknown of Eq. 4 (mu = h, delta = gamma h, sigma = 0); 0 = off."""
    _check(load_library().ei_set_linked(geom.handle, float(gamma)), "ei_set_linked")


def ei_offset_grad(geom: Geometry, vol, s_exp, g_mo=None, g_mr=None, stream=None):
    """dS/dm_o [sum n_theta] and dS/dm_r [sum n_det] (float32 device tensors,
    allocated when not given); returns (g_mo, g_mr)."""
    import torch
    n_th = sum(sl.n_theta for sl in geom.slices)
    n_px = sum(sl.n_det for sl in geom.slices)
    dev = vol.device
    if g_mo is None:
        g_mo = torch.empty(n_th, dtype=torch.float32, device=dev)
    if g_mr is None:
        g_mr = torch.empty(n_px, dtype=torch.float32, device=dev)
    _check_size(vol, geom.vol_count * 4, "vol")
    _check_size(s_exp, geom.meas_count, "s_exp")
    _check_size(g_mo, n_th, "g_mo")
    _check_size(g_mr, n_px, "g_mr")
    _check(load_library().ei_offset_grad(geom.handle, _dptr(vol, "vol"), _dptr(s_exp, "s_exp"),
                                         _dptr(g_mo, "g_mo"), _dptr(g_mr, "g_mr"),
                                         _stream_ptr(stream)), "ei_offset_grad")
    return g_mo, g_mr


def ei_measure_peaks(stream=None) -> dict:
    """On-chip throughput of the current GPU (FP32 FMA TFLOP/s, L1 and shared
    memory load TB/s), measured by microbenchmarks."""
    p = ei_peaks()
    _check(load_library().ei_measure_peaks(ctypes.byref(p), _stream_ptr(stream)), "ei_measure_peaks")
    return {f: getattr(p, f) for f, _ in p._fields_}


def ei_set_ic_variant(geom: Geometry, variant: int) -> None:
    """IC kernel variant: 0 one block per row, 1 persistent bulk-copy pipeline."""
    _check(load_library().ei_set_ic_variant(geom.handle, int(variant)), "ei_set_ic_variant")


def ei_get_ic_variant(geom: Geometry) -> int:
    v = c_int()
    _check(load_library().ei_get_ic_variant(geom.handle, ctypes.byref(v)), "ei_get_ic_variant")
    return v.value


class UNet:
    """The learned warm start's network (see include/ei.h: ei_unet_*).
    Arrays are FP32 CUDA tensors NHWC [batch][height][width][3]."""

    def __init__(self, levels: int = 4, base: int = 32, batch: int = 16, height: int = 256,
                 width: int = 256, seed: int = 0):
        h = c_void_p()
        _check(load_library().ei_unet_create(int(levels), int(base), int(batch), int(height),
                                             int(width), int(seed), ctypes.byref(h)),
               "ei_unet_create")
        self.handle = h.value
        self.levels, self.base, self.batch, self.height, self.width = levels, base, batch, height, width
        self.num_params = int(load_library().ei_unet_num_params(self.handle))

    def close(self):
        if self.handle:
            load_library().ei_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_io(self, t, name):
        import torch
        if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 4 or t.shape[1:] != (
                self.height, self.width, 3) or t.shape[0] > self.batch:
            raise ValueError("%s must be a CUDA float32 tensor [<=%d][%d][%d][3]"
                             % (name, self.batch, self.height, self.width))
        return _dptr(t, name)

    def forward(self, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(load_library().ei_unet_forward(self.handle, self._check_io(x, "x"),
                                              self._check_io(y, "y"), int(x.shape[0]),
                                              _stream_ptr(stream)), "ei_unet_forward")
        return y

    def train_step(self, x, target, lr: float, stream=None) -> float:
        loss = c_double()
        _check(load_library().ei_unet_train_step(self.handle, self._check_io(x, "x"),
                                                 self._check_io(target, "target"), int(x.shape[0]),
                                                 float(lr), ctypes.byref(loss), _stream_ptr(stream)),
               "ei_unet_train_step")
        return loss.value

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params, np.float32)
        _check(load_library().ei_unet_get_params(self.handle, out.ctypes.data), "ei_unet_get_params")
        return out

    def set_params(self, flat) -> None:
        arr = np.ascontiguousarray(flat, dtype=np.float32)
        if arr.size != self.num_params:
            raise ValueError("expected %d parameters" % self.num_params)
        _check(load_library().ei_unet_set_params(self.handle, arr.ctypes.data), "ei_unet_set_params")

    def set_tensor_path(self, path: int) -> None:
        """1: tcgen05 convolutions (default), 0: WMMA mma.sync."""
        _check(load_library().ei_unet_set_tensor_path(self.handle, int(path)), "ei_unet_set_tensor_path")

    def get_optimizer(self):
        """Adam's (m, v, step) for a training checkpoint."""
        m = np.empty(self.num_params, np.float32)
        v = np.empty(self.num_params, np.float32)
        step = c_int(0)
        _check(load_library().ei_unet_get_optimizer(self.handle, m.ctypes.data, v.ctypes.data,
                                                    ctypes.byref(step)), "ei_unet_get_optimizer")
        return m, v, step.value

    def set_optimizer(self, m, v, step: int) -> None:
        m = np.ascontiguousarray(m, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        if m.size != self.num_params or v.size != self.num_params:
            raise ValueError("optimizer state must have num_params entries")
        _check(load_library().ei_unet_set_optimizer(self.handle, m.ctypes.data, v.ctypes.data,
                                                    int(step)), "ei_unet_set_optimizer")

    def get_grads(self) -> np.ndarray:
        out = np.empty(self.num_params, np.float32)
        _check(load_library().ei_unet_get_grads(self.handle, out.ctypes.data), "ei_unet_get_grads")
        return out
