"""md_forces_noalloc: the entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc -- work enqueued during CUDA graph
capture, real-time loops and plugins that must not trigger the allocator or
its synchronisation, hosts with a fixed memory budget. md_forces_noalloc
serves them from one static device array. These tests call it through the C
ABI and check it against the FP64 CPU oracle (and, on two calls in a row,
against md_forces), within the FP64 force tolerance of the parity tests:

* boxes of 5 and 3 cells per edge (27-cell search), two calls in a row, so the
  second call starts from the first call's leftover scratch;
* a box too small for 3 cells per edge (N = 250 at density 1.2: all pairs);
* a dilute box of 36 cutoffs per edge, clamped to 32 cells per edge (the
  scratch holds at most 32^3 cells);
* n = 131072, the largest size the scratch takes (512 blocks fill its
  partial-sum array exactly): a melted N = 2048 liquid tiled 4 x 4 x 4, whose
  forces are the tiled oracle forces of the small box (r_c < L_2048 / 2);
* a type outside [0, ntypes), which must give NaN rather than read past the
  parameter table.

The file is collected last (its name), and it also passes on its own in a
fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_2001_07089_gb300 import kamd
from paper_2001_07089_gb300 import workloads as wl
from tests.helpers import force_errors, ka_params, melted

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


def _noalloc(pos, types, L, ntypes=2):
    import torch
    n = len(pos)
    dpos = torch.tensor(pos, dtype=torch.float64, device="cuda")
    dtyp = torch.tensor(np.asarray(types, dtype=np.uint8), device="cuda")
    f = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    pe = torch.zeros(1, dtype=torch.float64, device="cuda")
    vir = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    kamd.md_forces_noalloc(n, dpos, dtyp, ntypes, L, wl.KA_EPS[:ntypes, :ntypes], wl.KA_SIG[:ntypes, :ntypes],
                           wl.KA_RC[:ntypes, :ntypes], f, pe, vir, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return f.cpu().numpy(), float(pe.item()), float(vir.item())


def _check(f, pe, vir, f_ref, pe_ref, vir_ref):
    emax, e2 = force_errors(f, f_ref)
    assert emax <= TOL and e2 <= TOL, (emax, e2)
    assert abs(pe - pe_ref) <= TOL * abs(pe_ref)
    assert abs(vir - vir_ref) <= 10 * TOL * abs(vir_ref)


def test_noalloc_forces_match_oracle_and_md_forces_two_calls_in_a_row():
    cases = [melted(4000, 23, nsteps=200), melted(1000, 22, nsteps=200)]
    for pos, vel, types, L in cases:
        f_ora, pe_ora, vir_ora = oracle.forces(pos, types, ka_params(), L)
        f_ref, pe_ref, vir_ref = _reference(pos, vel, types, L)
        f, pe, vir = _noalloc(pos, types, L)
        _check(f, pe, vir, f_ora, pe_ora, vir_ora)
        _check(f, pe, vir, f_ref, pe_ref[0], vir_ref[0])


def test_noalloc_all_pairs_box():
    """N = 250 at density 1.2: L = 5.93 holds fewer than 3 cutoffs, so every pair is visited."""
    pos, vel, types, L = melted(250, 21, nsteps=200)
    assert L < 3 * wl.KA_RC.max()
    f_ora, pe_ora, vir_ora = oracle.forces(pos, types, ka_params(), L)
    _check(*_noalloc(pos, types, L), f_ora, pe_ora, vir_ora)


def test_noalloc_cell_clamp_dilute_box():
    """L = 90 would allow 36 cells of edge 2.5 per side; the scratch takes 32, so cells grow to 2.81."""
    n, L = 6000, 90.0
    assert int(L // wl.KA_RC.max()) > 32
    pos = wl.uniform_positions(n, L, 97)
    types = wl.ka_types(n, 97).astype(np.int32)
    f_ora, pe_ora, vir_ora = oracle.forces(pos, types, ka_params(), L)
    _check(*_noalloc(pos, types, L), f_ora, pe_ora, vir_ora)


def test_noalloc_largest_size_tiled_melt():
    """n = 131072 (the scratch maximum): a melted 2048-particle liquid tiled 4 x 4 x 4."""
    pos0, vel0, types0, L0 = melted(2048, 98, nsteps=100)
    assert wl.KA_RC.max() < 0.5 * L0
    k = np.arange(4)
    shifts = np.stack(np.meshgrid(k, k, k, indexing="ij"), axis=-1).reshape(-1, 3) * L0
    pos = np.concatenate([pos0 + s for s in shifts])
    types = np.concatenate([types0] * 64)
    L = 4 * L0
    assert len(pos) == 131072
    f0, pe0, vir0 = oracle.forces(pos0, types0, ka_params(), L0)
    f_ref = np.concatenate([f0] * 64)
    # the tiled reference is exact: spot-check it against O(N) sums of the big box
    for i in (0, 777, 65536, 131071):
        fi, _ = oracle.force_on(pos, types, ka_params(), L, i)
        assert np.max(np.abs(fi - f_ref[i])) < 1e-12 * max(1.0, np.abs(f0).max())
    f, pe, vir = _noalloc(pos, types, L)
    _check(f, pe, vir, f_ref, 64 * pe0, 64 * vir0)


def test_noalloc_out_of_range_type_gives_nan():
    """A type >= ntypes never indexes the tables: it turns its own force, those of the particles
    whose cell search meets it, and the energy and virial into NaN; the rest is unchanged."""
    pos, vel, types, L = melted(4000, 23, nsteps=200)
    w = L / int(L // wl.KA_RC.max())  # cell edge (5 cells per edge)
    bad = np.array(types, dtype=np.uint8)
    bad[17] = 2
    f, pe, vir = _noalloc(pos, bad, L)
    assert np.all(np.isnan(f[17])) and np.isnan(pe) and np.isnan(vir)
    f_ora, _, _ = oracle.forces(pos, types, ka_params(), L)
    d = pos - pos[17]
    d -= L * np.rint(d / L)
    far = np.any(np.abs(d) > 2 * w, axis=1)  # cells two or more apart along some axis
    ok = ~np.isnan(f[:, 0])
    assert far.sum() > 1000 and np.all(ok[far])
    frms = np.sqrt(np.mean(np.sum(f_ora * f_ora, axis=1)))
    assert np.max(np.linalg.norm(f[ok] - f_ora[ok], axis=1)) <= TOL * frms


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    n = 131073
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(kamd.KamdError) as ei:
        kamd.md_forces_noalloc(n, dummy, dummy, 2, 100.0, wl.KA_EPS, wl.KA_SIG, wl.KA_RC, dummy)
    assert ei.value.status == kamd.MD_ERR_INVALID_ARG
    assert "131072" in str(ei.value)
