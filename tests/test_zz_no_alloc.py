"""flip_solve_pressure_noalloc: the pressure solve for callers that cannot allocate.

Such callers (a plug-in whose device memory belongs to its host application's
allocator, or a latency-critical loop where cudaMalloc/cudaFree may not run because
they can synchronise the device) get the same solve from a fixed scratch array the
library owns.  This test calls the allocation-free entry point through the C ABI
several times in a row, on different inputs, and checks each result against the
allocating entry point flip_solve_pressure within the solver tests' tolerance
(relative L2 <= 1e-5).  The file is named to be collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="needs a CUDA GPU")]


def _case(n, seed):
    from paper_2404_01931_gb300 import flip as F
    from paper_2404_01931_gb300 import scenes as S
    t = S.random_mask(n, 0.7, seed).astype(np.uint8)
    rng = np.random.default_rng(seed)
    b = (rng.normal(size=t.shape) * t).astype(np.float32)
    fp = F.default_params(*n)
    fp.dx = 1.0 / max(n)
    fp.cg_tol = 1e-7
    return fp, torch.from_numpy(t.ravel()).cuda(), torch.from_numpy(b.ravel()).cuda()


def test_noalloc_solve_matches_allocating_solve_on_consecutive_calls():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2404_01931_gb300 import flip as F

    cases = [((13, 9, 11), 3), ((32, 40, 24), 4), ((13, 9, 11), 5), ((64, 64, 64), 6)]
    for n, seed in cases:
        fp, td, bd = _case(n, seed)
        ref = torch.full((td.numel(),), 3.0, dtype=torch.float32, device="cuda")
        got = torch.full((td.numel(),), -5.0, dtype=torch.float32, device="cuda")
        rc0, it0, rel0 = F.flip_solve_pressure(fp, td, bd, ref)
        rc1, it1, rel1 = F.flip_solve_pressure_noalloc(fp, td, bd, got)
        assert rc0 == F.FLIP_OK and rc1 == F.FLIP_OK
        assert it1 > 0 and rel1 <= 1e-7
        r, g = ref.cpu().numpy().astype(np.float64), got.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert err <= 1e-5, f"{n}: relative L2 {err:.3e}"
        assert np.all(g[td.cpu().numpy() == 0] == 0.0)


def test_noalloc_refuses_grids_beyond_its_scratch():
    from paper_2404_01931_gb300 import flip as F
    n = (65, 64, 64)  # 266,240 cells > FLIP_NOALLOC_MAX_CELLS
    fp = F.default_params(*n)
    td = torch.zeros(np.prod(n), dtype=torch.uint8, device="cuda")
    bd = torch.zeros(np.prod(n), dtype=torch.float32, device="cuda")
    pd = torch.zeros(np.prod(n), dtype=torch.float32, device="cuda")
    with pytest.raises(F.FlipError) as ei:
        F.flip_solve_pressure_noalloc(fp, td, bd, pd)
    assert ei.value.code == F.FLIP_E_SIZE and "exceeds" in str(ei.value)
