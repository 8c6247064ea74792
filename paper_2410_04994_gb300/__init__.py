"""GB300 split-step Fourier SHG library: thin Python binding of libshg.so.

Every function named ``shg_*`` here marshals its arguments and calls the C
entry point of the same name declared in ``include/shg.h``; all arithmetic of
the propagation runs in the library's CUDA kernels.  PyTorch supplies device
memory (tensors whose ``data_ptr`` is passed through) and streams.

The library is built in-tree by :func:`paper_2410_04994_gb300.build.build`;
loading fails loudly if it is missing, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libshg.so")

SHG_OK = 0
SHG_ERR_INVALID_ARG = 1
SHG_ERR_UNSUPPORTED_GRID = 2
SHG_ERR_OOM = 3
SHG_ERR_CUDA = 4
SHG_ERR_TIMEOUT = 5
SHG_ERR_NONFINITE = 6
SHG_ERR_STATE = 7

SHG_FLAG_FP64 = 1
SHG_FLAG_THERMAL = 2
SHG_FLAG_ADJOINT = 4
SHG_FLAG_NODE_SAMPLER = 8

SHG_FACE_OVEN = 0
SHG_FACE_CONVECTIVE = 1
SHG_HEAT_DIRECT = 0
SHG_HEAT_SOR = 1


class shg_grid_t(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double),
                ("hx", ctypes.c_int), ("hy", ctypes.c_int), ("hz", ctypes.c_int)]


class shg_crystal_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "L", "lambda_f", "n_f", "n_sh", "d_eff", "alpha_f", "alpha_sh", "beta_f", "beta_sh",
        "dk0", "ddk_dT", "dn_dT", "kappa_th", "wx", "wy", "walkoff_f", "walkoff_sh")]


class shg_beams_t(ctypes.Structure):
    _fields_ = [("p1", ctypes.c_double), ("w0", ctypes.c_double), ("z_focus", ctypes.c_double),
                ("t_oven_offset", ctypes.c_double), ("undepleted", ctypes.c_int)]


class shg_qpm_t(ctypes.Structure):
    _fields_ = [("t_oven", ctypes.c_double), ("lambda25", ctypes.c_double),
                ("a_lambda", ctypes.c_double), ("b_lambda", ctypes.c_double),
                ("n_f", ctypes.c_double * 4), ("n_sh", ctypes.c_double * 4)]


class shg_crystal3_t(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("lambda1", ctypes.c_double), ("lambda2", ctypes.c_double),
                ("n1", ctypes.c_double), ("n2", ctypes.c_double), ("n3", ctypes.c_double),
                ("d_eff", ctypes.c_double), ("alpha", ctypes.c_double * 3),
                ("beta", ctypes.c_double * 3), ("dk0", ctypes.c_double), ("ddk_dT", ctypes.c_double),
                ("dn_dT", ctypes.c_double), ("walkoff", ctypes.c_double * 3)]


class shg_beams3_t(ctypes.Structure):
    _fields_ = [("p", ctypes.c_double * 3), ("w0", ctypes.c_double * 3),
                ("z_focus", ctypes.c_double * 3), ("t_oven_offset", ctypes.c_double),
                ("undepleted", ctypes.c_int)]


class ShgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib().shg_status_string(status).decode()
        detail = _lib().shg_last_error().decode()
        super().__init__(f"{where}: {msg}" + (f" ({detail})" if detail else ""))


_LIB: Optional[ctypes.CDLL] = None

_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
_SIGS = {
    "shg_plan_create": [ctypes.POINTER(shg_grid_t), ctypes.POINTER(shg_crystal_t),
                        ctypes.POINTER(shg_beams_t), _I, ctypes.POINTER(_P)],
    "shg_plan_destroy": [_P],
    "shg_set_wait_limit": [_P, ctypes.c_uint],
    "shg_set_temperature_batch": [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), _I, _I, _I, _DP,
                                  _DP, _P],
    "shg_set_beams": [_P, ctypes.POINTER(shg_beams_t)],
    "shg_set_temperature": [_P, _P, _I, _I, _I, _D, _D, _P],
    "shg_set_fields": [_P, _P, _P, _P],
    "shg_propagate": [_P, _P],
    "shg_efficiency": [_P, _DP, _DP, _DP],
    "shg_get_fields": [_P, _P, _P, _P],
    "shg_propagate_adjoint": [_P, _D, _DP, _DP, _DP, _P, _P],
    "shg_batch_submit": [ctypes.POINTER(_P), _I, _DP, _P],
    "shg_heat_solve": [_P, _I, _D, _DP, _IP, _P],
    "shg_thermal_loop": [_P, _I, _I, _D, _DP, _DP, _P],
    "shg_get_heat": [_P, _P, _P, _P],
    "shg_pass_times": [ctypes.POINTER(_P), _I, _I, _DP, _IP, _I, _IP, _P],
    "shg_field_powers_noalloc": [_P, _I, _I, _I, _I, _D, _D, _D, _D, _P, _P],
    "shg_measure_peaks": [_DP, _DP, _DP, _DP, _P],
    "shg_set_monitor": [_P, _I],
    "shg_set_heat_boundary": [_P, _IP, _DP, _D],
    "shg_set_heat_method": [_P, _I],
    "shg_set_phase_model": [_P, ctypes.POINTER(shg_qpm_t)],
    "shg_plan_create_3w": [ctypes.POINTER(shg_grid_t), ctypes.POINTER(shg_crystal3_t),
                           ctypes.POINTER(shg_beams3_t), _I, ctypes.POINTER(_P)],
    "shg_get_field": [_P, _I, _P, _P],
    "shg_powers": [_P, _DP, _I],
    "shg_get_monitor": [_P, _DP, _DP, _DP, _I, _IP],
}
EXPORTED = list(_SIGS) + ["shg_status_string", "shg_last_error"]


def _lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2410_04994_gb300.build.build() "
                              "(nvcc, sm_103a); there is no fallback path")
        lib = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.shg_status_string.argtypes = [ctypes.c_int]
        lib.shg_status_string.restype = ctypes.c_char_p
        lib.shg_last_error.argtypes = []
        lib.shg_last_error.restype = ctypes.c_char_p
        _LIB = lib
    return _LIB


def load():
    """Load libshg.so (raises ImportError if it has not been built)."""
    return _lib()


def _check(status: int, where: str) -> None:
    if status != SHG_OK:
        raise ShgError(status, where)


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _map_shape(t):
    """(tz, ty, tx) of a temperature map; the library reads tz*ty*tx floats
    from its pointer, so anything but a 3-D float32 tensor is refused here."""
    import torch
    if not isinstance(t, torch.Tensor) or t.dim() != 3 or t.dtype != torch.float32:
        raise ValueError("a temperature map is a 3-D float32 tensor [tz][ty][tx]")
    if min(t.shape) < 2:
        raise ValueError("a temperature map has at least 2 nodes per axis")
    return tuple(t.shape)


def _field_check(t, nx: int, ny: int, fp64: bool) -> None:
    """A field handed to the library is read as ny*nx complex values of the
    plan's precision: refuse anything else."""
    import torch
    if t is None:
        return
    want = torch.complex128 if fp64 else torch.complex64
    if not isinstance(t, torch.Tensor) or t.dtype != want or t.numel() != nx * ny:
        raise ValueError(f"a field of this plan is a {want} tensor of {ny} x {nx} values")


# ------------------------------------------------- C entry points ----

def shg_plan_create(grid: shg_grid_t, crystal: shg_crystal_t, beams: shg_beams_t,
                    flags: int = 0) -> int:
    out = _P()
    _check(_lib().shg_plan_create(ctypes.byref(grid), ctypes.byref(crystal), ctypes.byref(beams),
                                  int(flags), ctypes.byref(out)), "shg_plan_create")
    return out.value


def shg_plan_destroy(plan: int) -> None:
    _check(_lib().shg_plan_destroy(plan), "shg_plan_destroy")


def shg_set_wait_limit(plan: int, polls: int) -> None:
    _check(_lib().shg_set_wait_limit(plan, int(polls)), "shg_set_wait_limit")


def shg_set_beams(plan: int, beams: shg_beams_t) -> None:
    _check(_lib().shg_set_beams(plan, ctypes.byref(beams)), "shg_set_beams")


def shg_set_temperature(plan: int, dT, t_lx: float = 0.0, t_ly: float = 0.0, stream=None) -> None:
    """dT: contiguous float32 CUDA tensor [tz][ty][tx], or None to clear.  A map
    of the installed shape and extent is copied asynchronously on `stream`:
    keep dT alive and unchanged until that stream has passed this call (with
    another stream than the one dT was allocated on, dT.record_stream(stream)
    keeps PyTorch's allocator from reusing it earlier)."""
    if dT is None:
        _check(_lib().shg_set_temperature(plan, None, 0, 0, 0, 0.0, 0.0, _stream(stream)),
               "shg_set_temperature")
        return
    tz, ty, tx = _map_shape(dT)
    _check(_lib().shg_set_temperature(plan, _ptr(dT), tx, ty, tz, float(t_lx), float(t_ly),
                                      _stream(stream)), "shg_set_temperature")


def shg_set_temperature_batch(plans: Sequence[int], maps, t_lx, t_ly, stream=None) -> None:
    """maps: contiguous float32 CUDA tensors [tz][ty][tx] of one shape, one per
    plan.  They are read asynchronously on `stream`, so they must stay alive
    and unchanged until that stream has passed this call (as for
    shg_set_temperature)."""
    n = len(plans)
    if n == 0 or len(maps) != n or len(t_lx) != n or len(t_ly) != n:
        raise ValueError("one map and one extent per plan")
    shapes = {_map_shape(m) for m in maps}
    if len(shapes) != 1:
        raise ValueError(f"the maps of one batch update share one shape, got {sorted(shapes)}")
    tz, ty, tx = shapes.pop()
    arr = (_P * n)(*plans)
    ptrs = (_P * n)(*[_ptr(m) for m in maps])
    lx = (_D * n)(*[float(v) for v in t_lx])
    ly = (_D * n)(*[float(v) for v in t_ly])
    _check(_lib().shg_set_temperature_batch(arr, n, ptrs, tx, ty, tz, lx, ly, _stream(stream)),
           "shg_set_temperature_batch")


def shg_set_fields(plan: int, a_f=None, a_sh=None, stream=None) -> None:
    _check(_lib().shg_set_fields(plan, _ptr(a_f), _ptr(a_sh), _stream(stream)), "shg_set_fields")


def shg_propagate(plan: int, stream=None) -> None:
    _check(_lib().shg_propagate(plan, _stream(stream)), "shg_propagate")


def shg_efficiency(plan: int):
    eta, pf, psh = _D(), _D(), _D()
    _check(_lib().shg_efficiency(plan, ctypes.byref(eta), ctypes.byref(pf), ctypes.byref(psh)),
           "shg_efficiency")
    return eta.value, pf.value, psh.value


def shg_get_fields(plan: int, a_f=None, a_sh=None, stream=None) -> None:
    _check(_lib().shg_get_fields(plan, _ptr(a_f), _ptr(a_sh), _stream(stream)), "shg_get_fields")


def shg_propagate_adjoint(plan: int, d_eta: float = 1.0, g_dT=None, stream=None):
    gw, gz, gt = _D(), _D(), _D()
    _check(_lib().shg_propagate_adjoint(plan, float(d_eta), ctypes.byref(gw), ctypes.byref(gz),
                                        ctypes.byref(gt), _ptr(g_dT), _stream(stream)),
           "shg_propagate_adjoint")
    return gw.value, gz.value, gt.value


def shg_batch_submit(plans: Sequence[int], stream=None):
    n = len(plans)
    arr = (_P * n)(*plans)
    etas = (_D * n)()
    _check(_lib().shg_batch_submit(arr, n, etas, _stream(stream)), "shg_batch_submit")
    return list(etas)


def shg_heat_solve(plan: int, max_sweeps: int = 100000, tol: float = 1e-6, stream=None):
    resid, sweeps = _D(), _I()
    _check(_lib().shg_heat_solve(plan, int(max_sweeps), float(tol), ctypes.byref(resid),
                                 ctypes.byref(sweeps), _stream(stream)), "shg_heat_solve")
    return resid.value, sweeps.value


def shg_thermal_loop(plan: int, n_outer: int, max_sweeps: int = 100000, tol: float = 1e-6,
                     stream=None):
    etas = (_D * n_outer)()
    changes = (_D * n_outer)()
    _check(_lib().shg_thermal_loop(plan, int(n_outer), int(max_sweeps), float(tol), etas, changes,
                                   _stream(stream)), "shg_thermal_loop")
    return list(etas), list(changes)


def shg_get_heat(plan: int, q=None, dT=None, stream=None) -> None:
    _check(_lib().shg_get_heat(plan, _ptr(q), _ptr(dT), _stream(stream)), "shg_get_heat")


def shg_pass_times(plans: Sequence[int], nsteps: int = 4, stream=None, max_groups: int = 16):
    """Average row/column pass launch times per grid group (CUDA events), and
    the group's schedule: passes_per_step 1 (row- and column-layout step
    passes alternate) or 2 (row pass, column pass)."""
    n = len(plans)
    arr = (_P * n)(*plans)
    out = (_D * (5 * max_groups))()
    inst = (_I * max_groups)()
    ng = _I()
    _check(_lib().shg_pass_times(arr, n, int(nsteps), out, inst, max_groups, ctypes.byref(ng),
                                 _stream(stream)), "shg_pass_times")
    return [dict(nx=int(out[5 * g]), ny=int(out[5 * g + 1]), row_ms=out[5 * g + 2],
                 col_ms=out[5 * g + 3], passes_per_step=int(out[5 * g + 4]), instances=inst[g])
            for g in range(ng.value)]


def shg_field_powers_noalloc(fields, nx: int, ny: int, n_inst: int, lx: float, ly: float,
                             n_f: float, n_sh: float, powers, stream=None) -> None:
    """P_F, P_SH of caller-held fields into a caller-held float64 CUDA tensor
    [n_inst, 2]; the library allocates nothing (see include/shg.h).

    The library reads n_inst * 2 * ny * nx complex values from `fields` and
    writes 2 * n_inst doubles to `powers`, so any tensor it would read or
    write past its end, or reinterpret as another type, is refused here
    (ValueError) before the call."""
    import torch
    if not isinstance(fields, torch.Tensor) or fields.dtype not in (torch.complex64,
                                                                   torch.complex128):
        raise ValueError("fields is a complex64 or complex128 tensor")
    if not isinstance(powers, torch.Tensor) or powers.dtype != torch.float64:
        raise ValueError("powers is a float64 tensor")
    n_inst, nx, ny = int(n_inst), int(nx), int(ny)
    if n_inst < 1 or nx < 1 or ny < 1 or fields.numel() != n_inst * 2 * nx * ny:
        raise ValueError(f"fields holds {fields.numel()} values, not n_inst x 2 x ny x nx = "
                         f"{n_inst} x 2 x {ny} x {nx}")
    if powers.numel() < 2 * n_inst:
        raise ValueError(f"powers holds {powers.numel()} values, fewer than 2 x n_inst")
    for t in (fields, powers):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("fields and powers are contiguous CUDA tensors")
        if t.device.index != torch.cuda.current_device():
            raise ValueError("fields and powers live on the current CUDA device")
    fp64 = 1 if fields.dtype == torch.complex128 else 0
    _check(_lib().shg_field_powers_noalloc(_ptr(fields), nx, ny, n_inst, fp64, float(lx),
                                           float(ly), float(n_f), float(n_sh), _ptr(powers),
                                           _stream(stream)), "shg_field_powers_noalloc")


def shg_set_heat_boundary(plan: int, kinds, h=None, t_inf: float = 0.0) -> None:
    """kinds: six of SHG_FACE_OVEN / SHG_FACE_CONVECTIVE ("D" / "C" accepted) for
    the faces x-, x+, y-, y+, z-, z+; h: one coefficient or six (W/(m^2 K))."""
    if len(kinds) != 6:
        raise ValueError("six faces: x-, x+, y-, y+, z-, z+")
    code = {"D": SHG_FACE_OVEN, "C": SHG_FACE_CONVECTIVE}
    k = (_I * 6)(*[code.get(v, v) if isinstance(v, str) else int(v) for v in kinds])
    hv = [float(h or 0.0)] * 6 if not isinstance(h, (list, tuple)) else [float(v) for v in h]
    if len(hv) != 6:
        raise ValueError("one heat transfer coefficient or six")
    _check(_lib().shg_set_heat_boundary(plan, k, (_D * 6)(*hv), float(t_inf)),
           "shg_set_heat_boundary")


def shg_set_heat_method(plan: int, method: int) -> None:
    _check(_lib().shg_set_heat_method(plan, int(method)), "shg_set_heat_method")


def shg_plan_create_3w(grid: shg_grid_t, crystal: shg_crystal3_t, beams: shg_beams3_t,
                       flags: int = 0) -> int:
    out = _P()
    _check(_lib().shg_plan_create_3w(ctypes.byref(grid), ctypes.byref(crystal), ctypes.byref(beams),
                                     int(flags), ctypes.byref(out)), "shg_plan_create_3w")
    return out.value


def shg_get_field(plan: int, j: int, dev, stream=None) -> None:
    _check(_lib().shg_get_field(plan, int(j), _ptr(dev), _stream(stream)), "shg_get_field")


def shg_powers(plan: int, n: int = 3):
    out = (_D * n)()
    _check(_lib().shg_powers(plan, out, int(n)), "shg_powers")
    return list(out)


def shg_set_phase_model(plan: int, qpm=None) -> None:
    """Eq. (4) phase model from an object with t_oven, lambda25, a_lambda,
    b_lambda, n_f_t, n_sh_t (index polynomials in T - 25 C, up to cubic), or
    None for the linearised model."""
    if qpm is None:
        _check(_lib().shg_set_phase_model(plan, None), "shg_set_phase_model")
        return
    nf, ns = list(qpm.n_f_t), list(qpm.n_sh_t)
    if len(nf) > 4 or len(ns) > 4:
        raise ValueError("index polynomials of degree 3 at most")
    m = shg_qpm_t(float(qpm.t_oven), float(qpm.lambda25), float(qpm.a_lambda),
                  float(qpm.b_lambda), (ctypes.c_double * 4)(*(nf + [0.0] * (4 - len(nf)))),
                  (ctypes.c_double * 4)(*(ns + [0.0] * (4 - len(ns)))))
    _check(_lib().shg_set_phase_model(plan, ctypes.byref(m)), "shg_set_phase_model")


def shg_set_monitor(plan: int, every: int) -> None:
    _check(_lib().shg_set_monitor(plan, int(every)), "shg_set_monitor")


def shg_get_monitor(plan: int):
    """(z, P_F, P_SH) lists of the power monitor's samples of the last
    propagation (see include/shg.h)."""
    n = _I()
    _check(_lib().shg_get_monitor(plan, None, None, None, 0, ctypes.byref(n)), "shg_get_monitor")
    z, pf, psh = (_D * n.value)(), (_D * n.value)(), (_D * n.value)()
    _check(_lib().shg_get_monitor(plan, z, pf, psh, n.value, ctypes.byref(n)), "shg_get_monitor")
    return list(z), list(pf), list(psh)


def shg_measure_peaks(stream=None):
    """Measured FP32 FMA throughput (packed and scalar), FP64 FMA throughput
    (TFLOP/s) and L2 read bandwidth (GB/s) of the current device."""
    f, l2, fs, f64 = _D(), _D(), _D(), _D()
    _check(_lib().shg_measure_peaks(ctypes.byref(f), ctypes.byref(l2), ctypes.byref(fs),
                                    ctypes.byref(f64), _stream(stream)), "shg_measure_peaks")
    return {"fp32_tflops": f.value, "fp32_scalar_tflops": fs.value, "fp64_tflops": f64.value,
            "l2_read_gbs": l2.value}


def shg_status_string(status: int) -> str:
    return _lib().shg_status_string(status).decode()


# ------------------------------------------------------ conveniences ----

def structs_from(w, flags: int = 0):
    """(grid, crystal, beams) structs from any object with the workload fields
    (nx, ny, nz, lx, ly, L, lambda_f, ..., p1, w0, z_focus, t_off, undepleted)."""
    grid = shg_grid_t(w.nx, w.ny, w.nz, w.lx, w.ly, getattr(w, "hx", 0), getattr(w, "hy", 0),
                      getattr(w, "hz", 0))
    crystal = shg_crystal_t(w.L, w.lambda_f, w.n_f, w.n_sh, w.d_eff, w.alpha_f, w.alpha_sh,
                            w.beta_f, w.beta_sh, w.dk0, w.ddk_dT, w.dn_dT, w.kappa_th, w.wx, w.wy,
                            getattr(w, "walkoff_f", 0.0), getattr(w, "walkoff_sh", 0.0))
    beams = shg_beams_t(w.p1, w.w0, w.z_focus, w.t_off, 1 if w.undepleted else 0)
    return grid, crystal, beams


class Plan:
    """Owning handle around an shg plan (destroyed with the object)."""

    def __init__(self, w, flags: Optional[int] = None, thermal: bool = False,
                 adjoint: bool = False, node_sampler: bool = False):
        if flags is None:
            flags = SHG_FLAG_FP64 if getattr(w, "precision", "f32") == "f64" else 0
            if thermal:
                flags |= SHG_FLAG_THERMAL
            if adjoint:
                flags |= SHG_FLAG_ADJOINT
            if node_sampler:
                flags |= SHG_FLAG_NODE_SAMPLER
        self.w = w
        self.flags = flags
        self.fp64 = bool(flags & SHG_FLAG_FP64)
        self.handle = shg_plan_create(*structs_from(w), flags)
        self._dT = None
        if getattr(w, "qpm", None) is not None:
            shg_set_phase_model(self.handle, w.qpm)
        faces = tuple(getattr(w, "heat_faces", ("D",) * 6))
        if (flags & SHG_FLAG_THERMAL) and any(f != "D" for f in faces):
            shg_set_heat_boundary(self.handle, faces, getattr(w, "h_conv", 0.0),
                                  getattr(w, "t_inf", 0.0))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                shg_plan_destroy(h)
            except Exception:
                pass
            self.handle = None

    def set_temperature(self, dT, t_lx=0.0, t_ly=0.0, stream=None):
        import torch
        if dT is not None and not isinstance(dT, torch.Tensor):
            dT = torch.as_tensor(dT, dtype=torch.float32, device="cuda")
        if dT is not None:
            dT = dT.to(device="cuda", dtype=torch.float32).contiguous()
        self._dT = dT
        shg_set_temperature(self.handle, dT, t_lx, t_ly, stream)

    def set_beams(self, p1=None, w0=None, z_focus=None, t_off=None, undepleted=None):
        w = self.w
        b = shg_beams_t(w.p1 if p1 is None else p1, w.w0 if w0 is None else w0,
                        w.z_focus if z_focus is None else z_focus,
                        w.t_off if t_off is None else t_off,
                        int(w.undepleted if undepleted is None else undepleted))
        shg_set_beams(self.handle, b)

    def set_fields(self, a_f=None, a_sh=None, stream=None):
        for a in (a_f, a_sh):
            _field_check(a, self.w.nx, self.w.ny, self.fp64)
        shg_set_fields(self.handle, a_f, a_sh, stream)

    def propagate(self, stream=None):
        shg_propagate(self.handle, stream)

    def efficiency(self):
        return shg_efficiency(self.handle)

    def fields(self, stream=None):
        import torch
        dt = torch.complex128 if self.fp64 else torch.complex64
        a_f = torch.empty((self.w.ny, self.w.nx), dtype=dt, device="cuda")
        a_sh = torch.empty_like(a_f)
        shg_get_fields(self.handle, a_f, a_sh, stream)
        return a_f, a_sh


def structs3_from(w):
    """(grid, crystal, beams) structs of a three-wave workload (an object with
    nx, ny, nz, lx, ly, L, lambda1, lambda2, n1, n2, n3, d_eff, alpha, beta,
    dk0, ddk_dT, dn_dT, walkoff, p, w0, z_focus, t_off, undepleted)."""
    t3 = ctypes.c_double * 3
    grid = shg_grid_t(w.nx, w.ny, w.nz, w.lx, w.ly, 0, 0, 0)
    crystal = shg_crystal3_t(w.L, w.lambda1, w.lambda2, w.n1, w.n2, w.n3, w.d_eff, t3(*w.alpha),
                             t3(*w.beta), w.dk0, w.ddk_dT, w.dn_dT, t3(*w.walkoff))
    beams = shg_beams3_t(t3(*w.p), t3(*w.w0), t3(*w.z_focus), w.t_off, 1 if w.undepleted else 0)
    return grid, crystal, beams


class Plan3:
    """Owning handle around a three-wave (sum/difference-frequency) plan."""

    def __init__(self, w):
        self.w = w
        self.fp64 = getattr(w, "precision", "f32") == "f64"
        self.handle = shg_plan_create_3w(*structs3_from(w), SHG_FLAG_FP64 if self.fp64 else 0)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                shg_plan_destroy(h)
            except Exception:
                pass
            self.handle = None

    def set_temperature(self, dT, t_lx=0.0, t_ly=0.0, stream=None):
        import torch
        dT = torch.as_tensor(dT).to(device="cuda", dtype=torch.float32).contiguous()
        self._dT = dT
        shg_set_temperature(self.handle, dT, t_lx, t_ly, stream)

    def propagate(self, stream=None):
        shg_propagate(self.handle, stream)

    def powers(self):
        return shg_powers(self.handle, 3)

    def fields(self, stream=None):
        import torch
        dt = torch.complex128 if self.fp64 else torch.complex64
        out = []
        for j in range(3):
            a = torch.empty((self.w.ny, self.w.nx), dtype=dt, device="cuda")
            shg_get_field(self.handle, j, a, stream)
            out.append(a)
        return out
