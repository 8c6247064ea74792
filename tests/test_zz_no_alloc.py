"""The allocation-free power entry point against the plan's own reduction and
the oracle.

shg_field_powers_noalloc is for callers that may not allocate device memory
(a fixed memory budget owned by a host framework, or a latency-critical
loop): it works on caller-held fields and output and keeps its partial sums
in a static device array.  This file runs last so that a failure here leaves
every other test already run.
"""
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_powers_match_plan_reduction_twice():
    import paper_2410_04994_gb300 as pkg
    for w in (W.depleted_absorbing(n=64, nz=20, tgrid=(8, 8, 8), p1=200.0),
              W.plain_focused(n=32, nz=20)):          # FP32 then FP64 fields
        plan = pkg.Plan(w)
        if w.dT is not None:
            plan.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
        plan.propagate()
        eta, p_f, p_sh = plan.efficiency()
        a_f, a_sh = plan.fields()
        fields = torch.stack([a_f, a_sh]).contiguous()
        for _ in range(2):   # the shared scratch must not carry state between calls
            out = torch.full((1, 2), float("nan"), dtype=torch.float64, device="cuda")
            pkg.shg_field_powers_noalloc(fields, w.nx, w.ny, 1, w.lx, w.ly, w.n_f, w.n_sh, out)
            torch.cuda.synchronize()
            got_f, got_sh = float(out[0, 0]), float(out[0, 1])
            assert abs(got_f / p_f - 1) < 1e-12
            assert abs(got_sh / p_sh - 1) < 1e-12


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_noalloc_many_instances_match_the_oracle_power(dtype):
    """Several instances with different fields (scaled copies of one
    propagated pair, so every row differs): each row of the output equals
    the oracle's discrete power of that instance's fields, on two calls in
    a row; the second call uses fewer instances than the first, so a row
    left over from the first call cannot pass for a result."""
    import paper_2410_04994_gb300 as pkg
    from oracle import ssfm
    w = W.depleted_absorbing(n=64, nz=20, tgrid=(8, 8, 8), p1=200.0)
    plan = pkg.Plan(w)
    plan.set_temperature(torch.as_tensor(w.dT), w.t_lx, w.t_ly)
    plan.propagate()
    a_f, a_sh = plan.fields()
    base = torch.stack([a_f, a_sh]).to(dtype)
    scales = [1.0, 0.5, 2.0, 3.0, 0.25]
    dx, dy = w.lx / w.nx, w.ly / w.ny
    for n_inst in (5, 3):
        fields = torch.stack([s * base for s in scales[:n_inst]]).contiguous()
        out = torch.full((n_inst, 2), float("nan"), dtype=torch.float64, device="cuda")
        pkg.shg_field_powers_noalloc(fields, w.nx, w.ny, n_inst, w.lx, w.ly, w.n_f, w.n_sh, out)
        torch.cuda.synchronize()
        host = fields.cpu().to(torch.complex128)
        for k in range(n_inst):
            ref_f = float(ssfm.power(host[k, 0], w.n_f, dx, dy))
            ref_sh = float(ssfm.power(host[k, 1], w.n_sh, dx, dy))
            assert abs(float(out[k, 0]) / ref_f - 1) < 1e-12, (k, float(out[k, 0]), ref_f)
            assert abs(float(out[k, 1]) / ref_sh - 1) < 1e-12, (k, float(out[k, 1]), ref_sh)


def test_noalloc_refuses_more_instances_than_its_scratch_holds():
    """1025 instances of well-formed tensors pass the binding and are refused
    by the library (the static scratch holds 1024)."""
    import paper_2410_04994_gb300 as pkg
    n = 1025
    fields = torch.zeros((n, 2, 8, 8), dtype=torch.complex64, device="cuda")
    out = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.ShgError) as ei:
        pkg.shg_field_powers_noalloc(fields, 8, 8, n, 1e-3, 1e-3, 2.14, 2.18, out)
    assert ei.value.status == pkg.SHG_ERR_INVALID_ARG
