"""md_forces_noalloc: the entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc -- work enqueued during CUDA graph
capture, real-time loops and plugins that must not trigger the allocator or
its synchronisation, hosts with a fixed memory budget. md_forces_noalloc
serves them from one static device array. This test calls it through the C
ABI twice in a row (two different systems, so the second call starts from
the first call's leftover scratch) and checks each result against md_forces
on the FP64 path, within the FP64 force tolerance of the parity tests. It
runs last (file name) and also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2001_07089_gb300 import kamd
from paper_2001_07089_gb300 import workloads as wl
from tests.helpers import force_errors, melted

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kamd.load()


def _reference(pos, vel, types, L):
    with kamd.System(len(pos), L, types, wl.KA_EPS, wl.KA_SIG, wl.KA_RC, 1.0, 0.3, "fp64") as s:
        s.set_state(pos, vel)
        return s.forces()


def _noalloc(pos, types, L):
    import torch
    n = len(pos)
    dpos = torch.tensor(pos, dtype=torch.float64, device="cuda")
    dtyp = torch.tensor(np.asarray(types, dtype=np.uint8), device="cuda")
    f = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    pe = torch.zeros(1, dtype=torch.float64, device="cuda")
    vir = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    kamd.md_forces_noalloc(n, dpos, dtyp, 2, L, wl.KA_EPS, wl.KA_SIG, wl.KA_RC, f, pe, vir,
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return f.cpu().numpy(), float(pe.item()), float(vir.item())


def test_noalloc_forces_match_md_forces_two_calls_in_a_row():
    cases = [melted(4000, 23, nsteps=200), melted(1000, 22, nsteps=200)]
    for pos, vel, types, L in cases:
        f_ref, pe_ref, vir_ref = _reference(pos, vel, types, L)
        f, pe, vir = _noalloc(pos, types, L)
        emax, e2 = force_errors(f, f_ref)
        assert emax <= TOL and e2 <= TOL, (len(pos), emax, e2)
        assert abs(pe - pe_ref[0]) <= TOL * abs(pe_ref[0])
        assert abs(vir - vir_ref[0]) <= 10 * TOL * abs(vir_ref[0])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    n = 131073
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(kamd.KamdError) as ei:
        kamd.md_forces_noalloc(n, dummy, dummy, 2, 100.0, wl.KA_EPS, wl.KA_SIG, wl.KA_RC, dummy)
    assert ei.value.status == kamd.MD_ERR_INVALID_ARG
    assert "131072" in str(ei.value)
