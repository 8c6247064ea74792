"""Host-side checks of libshg.so that need no GPU: it loads, exports every
entry point declared in include/shg.h, and rejects bad arguments before any
device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2410_04994_gb300 import build
    build.build()
    import paper_2410_04994_gb300 as p
    p.load()
    return p


def declared():
    src = open(os.path.join(ROOT, "include", "shg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(shg_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(pkg):
    names = declared()
    assert len(names) >= 14
    lib = ctypes.CDLL(pkg.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(pkg.EXPORTED)


def test_status_strings(pkg):
    for code in range(8):
        assert pkg.shg_status_string(code) != "unknown status"
    assert pkg.shg_status_string(99) == "unknown status"


def _w(**kw):
    import workloads as W
    return W.plain_focused(n=32, nz=10, precision="f32").with_(**kw)


@pytest.mark.parametrize("kw,flags,code", [
    (dict(nx=12), 0, 2),
    (dict(ny=2048), 0, 2),
    (dict(nx=4), 0, 2),
    (dict(nx=512), 1, 2),
    (dict(nz=0), 0, 1),
    (dict(lx=0.0), 0, 1),
    (dict(w0=0.0), 0, 1),
    (dict(p1=-1.0), 0, 1),
    (dict(L=0.0), 0, 1),
    (dict(hx=2, hy=8, hz=8), 2, 1),
    (dict(hx=8, hy=8, hz=8, kappa_th=0.0), 2, 1),
    (dict(nz=(1 << 26) + 1), 0, 1),
    (dict(lx=float("inf")), 0, 1),
    (dict(d_eff=float("nan")), 0, 1),
    (dict(dn_dT=float("inf")), 0, 1),
    (dict(z_focus=float("nan")), 0, 1),
    (dict(t_off=float("-inf")), 0, 1),
    (dict(walkoff_sh=1.6), 0, 1),
    (dict(n_sh=0.0), 0, 1),
])
def test_plan_create_rejects_bad_arguments(pkg, kw, flags, code):
    w = _w(**kw)
    with pytest.raises(pkg.ShgError) as ei:
        pkg.shg_plan_create(*pkg.structs_from(w), flags)
    assert ei.value.status == code


def test_null_handles_are_rejected(pkg):
    lib = pkg.load()
    assert lib.shg_plan_create(None, None, None, 0, None) == 1
    assert lib.shg_plan_destroy(None) == 0
    assert lib.shg_propagate(None, None) == 1
    assert lib.shg_efficiency(None, None, None, None) == 1
    assert lib.shg_batch_submit(None, 0, None, None) == 1
    assert lib.shg_propagate_adjoint(None, 1.0, None, None, None, None, None) == 1
    assert lib.shg_heat_solve(None, 1, 1e-6, None, None, None) == 1
    assert lib.shg_thermal_loop(None, 1, 1, 1e-6, None, None, None) == 1
    assert lib.shg_get_heat(None, None, None, None) == 1
    assert lib.shg_set_wait_limit(None, 0) == 1
    assert lib.shg_set_beams(None, None) == 1
    assert lib.shg_set_temperature(None, None, 2, 2, 2, 0.0, 0.0, None) == 1
    assert lib.shg_set_temperature_batch(None, 0, None, 2, 2, 2, None, None, None) == 1
    assert lib.shg_set_fields(None, None, None, None) == 1
    assert lib.shg_get_fields(None, None, None, None) == 1
    assert lib.shg_pass_times(None, 0, 1, None, None, 1, None, None) == 1
    assert lib.shg_field_powers_noalloc(None, 8, 8, 1, 0, 1.0, 1.0, 2.0, 2.0, None, None) == 1


def test_missing_library_fails_loudly(pkg, monkeypatch, tmp_path):
    """Without libshg.so every entry point raises: there is no CPU or library
    fallback behind the binding."""
    import workloads as W
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "absent" / "libshg.so"))
    monkeypatch.setattr(pkg, "_LIB", None)
    with pytest.raises(ImportError, match="no fallback"):
        pkg.load()
    with pytest.raises(ImportError):
        pkg.Plan(W.plain_focused(n=8, nz=2))
    with pytest.raises(ImportError):
        pkg.shg_status_string(0)


def test_binding_refuses_maps_the_library_would_misread(pkg):
    """The library reads tz*ty*tx floats from each map pointer with one shape
    per batch: a map of another dtype, rank or shape is refused in the
    binding, before any pointer reaches the library."""
    import torch
    good = torch.zeros((4, 3, 5), dtype=torch.float32)
    bad = [torch.zeros((4, 3, 5), dtype=torch.float16), torch.zeros((4, 3, 5), dtype=torch.float64),
           torch.zeros((3, 5), dtype=torch.float32), torch.zeros((4, 1, 5), dtype=torch.float32)]
    for m in bad:
        with pytest.raises(ValueError, match="temperature map"):
            pkg.shg_set_temperature(0, m)
    with pytest.raises(ValueError, match="one shape"):
        pkg.shg_set_temperature_batch([0, 0], [good, torch.zeros((4, 3, 4))], [0.0, 0.0], [0.0, 0.0])
    with pytest.raises(ValueError, match="per plan"):
        pkg.shg_set_temperature_batch([0, 0], [good], [0.0], [0.0])


def test_binding_refuses_fields_of_another_size_or_precision(pkg):
    import torch
    ok32 = torch.zeros((8, 16), dtype=torch.complex64)
    pkg._field_check(ok32, 16, 8, False)
    pkg._field_check(torch.zeros((8, 16), dtype=torch.complex128), 16, 8, True)
    pkg._field_check(None, 16, 8, False)
    for t, fp64 in ((ok32, True), (torch.zeros((8, 8), dtype=torch.complex64), False),
                    (torch.zeros((8, 16, 2), dtype=torch.float32), False)):
        with pytest.raises(ValueError, match="field of this plan"):
            pkg._field_check(t, 16, 8, fp64)


def test_the_same_plan_twice_is_refused(pkg):
    """A plan listed twice in one multi-plan call would have two instances
    write its fields or tables at once; the call is refused before any plan
    is touched (the handle here is never dereferenced)."""
    import ctypes
    lib = pkg.load()
    fake = 0x1000
    arr = (ctypes.c_void_p * 2)(fake, fake)
    assert lib.shg_batch_submit(arr, 2, None, None) == 1
    maps = (ctypes.c_void_p * 2)(fake, fake)
    ext = (ctypes.c_double * 2)(0.0, 0.0)
    assert lib.shg_set_temperature_batch(arr, 2, maps, 2, 2, 2, ext, ext, None) == 1
    out = (ctypes.c_double * 10)()
    ng = ctypes.c_int()
    assert lib.shg_pass_times(arr, 2, 1, out, None, 2, ctypes.byref(ng), None) == 1


@pytest.mark.parametrize("case", ["real_fields", "short_fields", "long_fields", "f32_powers",
                                  "short_powers", "cpu_tensors", "bad_n_inst"])
def test_noalloc_binding_refuses_mismatched_tensors(pkg, case):
    """shg_field_powers_noalloc reads n_inst*2*ny*nx complex values and writes
    2*n_inst doubles: the binding refuses, before any library call, every
    tensor that the kernels would read or write past its end or reinterpret
    as another type."""
    import torch
    nx, ny, n = 8, 8, 3
    fields = torch.zeros((n, 2, ny, nx), dtype=torch.complex64)
    powers = torch.zeros((n, 2), dtype=torch.float64)
    kw = dict(n_inst=n)
    if case == "real_fields":
        fields = torch.zeros((n, 2, ny, nx, 2), dtype=torch.float64)
    elif case == "short_fields":
        fields = fields[:2]
    elif case == "long_fields":
        kw["n_inst"] = 2
        powers = powers[:2]
    elif case == "f32_powers":
        powers = powers.float()
    elif case == "short_powers":
        powers = powers[:2]
    elif case == "bad_n_inst":
        kw["n_inst"] = 0
    with pytest.raises(ValueError):
        pkg.shg_field_powers_noalloc(fields, nx, ny, kw["n_inst"], 1e-3, 1e-3, 2.14, 2.18,
                                     powers)


def test_refused_temperature_update_keeps_the_map(pkg):
    """Arguments are checked before the plan changes: a refused
    shg_set_temperature / shg_set_temperature_batch returns
    SHG_ERR_INVALID_ARG with no device work (no GPU needed to reach it)."""
    lib = pkg.load()
    # a NULL plan, and a non-NULL map with too few nodes, are refused first
    assert lib.shg_set_temperature(None, None, 0, 0, 0, 0.0, 0.0, None) == 1
    arr = (ctypes.c_void_p * 1)(1)   # never dereferenced: the shape check comes first
    maps = (ctypes.c_void_p * 1)(1)
    ext = (ctypes.c_double * 1)(0.0)
    assert lib.shg_set_temperature_batch(arr, 1, maps, 1, 4, 4, ext, ext, None) == 1
    bad = (ctypes.c_double * 1)(float("nan"))
    assert lib.shg_set_temperature_batch(arr, 1, maps, 4, 4, 4, bad, ext, None) == 1


def test_monitor_calls_refuse_bad_arguments(pkg):
    lib = pkg.load()
    assert lib.shg_set_monitor(None, 1) == 1
    assert lib.shg_get_monitor(None, None, None, None, 0, None) == 1
    assert lib.shg_measure_peaks(None, None, None, None, None) == 1


def test_heat_calls_refuse_null_plans(pkg):
    lib = pkg.load()
    kinds = (ctypes.c_int * 6)(0, 0, 0, 0, 0, 0)
    assert lib.shg_set_heat_boundary(None, kinds, None, 0.0) == 1
    assert lib.shg_set_heat_method(None, 0) == 1
