"""The allocation-free totals entry point (sif_integrals_noalloc) agrees
with the context's own sif_integrals on two calls in a row.

It exists for callers that cannot allocate device memory at the point
where they need the totals, e.g. a host framework whose caching allocator
already holds the GPU's free memory.  This file is collected last."""
import numpy as np
import pytest

from paper_1905_03917_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_totals_match_context_totals_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_03917_gb300 import sif
    case = inputs.periodic_bubble(48, seed=1)
    cfg = case["cfg"]
    s = sif.Solver(cfg).init_fluids(*(np.ascontiguousarray(case[x]) for x in ("phi", "prim_N", "prim_P")))
    ny, nx = cfg["ny"], cfg["nx"]
    qN = torch.empty((4, ny, nx), dtype=torch.float64, device="cuda")
    qP = torch.empty((4, ny, nx), dtype=torch.float64, device="cuda")
    phi = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        s.step_multi_dt(3)
        ref = s.integrals()
        s.state_into(qN, qP, phi)
        sif.integrals_noalloc(qN, qP, cfg["dx"], cfg["dy"], out)
        got = out.cpu().numpy().reshape(2, 4)
        assert np.all(np.isfinite(got))
        # both reductions take one warp per row, the same lane striding and
        # shuffle tree, the same row order and no FMA contraction: equal bits
        assert np.array_equal(got, ref), np.abs(got - ref).max()


def test_noalloc_rejects_rows_beyond_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_03917_gb300 import sif
    q = torch.zeros((4, 16385, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(sif.SifError) as e:
        sif.integrals_noalloc(q, q, 1.0, 1.0, out)
    assert e.value.code == sif.EINVAL


def test_noalloc_rejects_malformed_tensors():
    """Shapes that would make the kernels read or write past a buffer are
    refused in the binding before any launch."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_03917_gb300 import sif
    q = torch.zeros((4, 8, 8), dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        sif.integrals_noalloc(q[0], q[0], 1.0, 1.0, out)      # (ny, nx), not (4, ny, nx)
    with pytest.raises(ValueError):
        sif.integrals_noalloc(q, q[:, :4].contiguous(), 1.0, 1.0, out)  # q_P of another shape
    with pytest.raises(ValueError):
        sif.integrals_noalloc(q, q, 1.0, 1.0, out[:4])       # out too short
