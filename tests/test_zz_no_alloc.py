"""The allocation-free power entry point against the plan's own reduction.

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
    # more instances than the static scratch holds are refused
    with pytest.raises(pkg.ShgError) as ei:
        pkg.shg_field_powers_noalloc(fields, w.nx, w.ny, 1025, w.lx, w.ly, w.n_f, w.n_sh, out)
    assert ei.value.status == pkg.SHG_ERR_INVALID_ARG
