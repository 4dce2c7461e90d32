"""The reciprocal inside the finite-volume kernel's WENO5 face values
(Newton's iteration to third order from the device's approximate
reciprocal) against IEEE division on the host: within 1 ulp of the
correctly rounded 1/d over the whole input range the kernel uses it for
(positive normal d below 2^1000), at powers of two, just below them and at
the ends of the range."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs():
    rng = np.random.default_rng(20190509)
    n = 1 << 20
    m = 1.0 + rng.random(n)                       # [1, 2)
    e = rng.integers(-1021, 999, size=n)          # 2^-1021 .. 2^999
    d = np.ldexp(m, e)
    edges = [1.0, 2.0, 0.5, 3.0, 1.0 / 3.0, 0.1, 0.6, 0.3, 1e-6, 1e-12, 1e-50, 1e100, 1e200,
             np.nextafter(2.0, 0.0), np.nextafter(1.0, 0.0), np.nextafter(1.0, 2.0),
             np.ldexp(1.0, -1021), np.ldexp(1.0, 999), np.nextafter(np.ldexp(1.0, 1000), 0.0)]
    return np.concatenate([d, np.asarray(edges, dtype=np.float64)])


def test_reciprocal_within_one_ulp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_03917_gb300 import sif
    d = _inputs()
    assert np.all(d > 0) and np.all(d < 2.0 ** 1000) and np.all(d >= np.finfo(np.float64).tiny)
    r = sif.probe_reciprocal(torch.from_numpy(d).cuda())
    torch.cuda.synchronize()
    r = r.cpu().numpy()
    q = 1.0 / d
    ulp = np.abs(r.view(np.int64) - q.view(np.int64))
    print("max ulp", ulp.max(), "not correctly rounded", int((ulp != 0).sum()), "of", d.size)
    assert ulp.max() <= 1
    # exact where the reciprocal is a power of two
    p2 = np.ldexp(1.0, np.arange(-1000, 999))
    r2 = sif.probe_reciprocal(torch.from_numpy(p2).cuda()).cpu().numpy()
    assert np.array_equal(r2, 1.0 / p2)


def test_reciprocal_arguments():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_03917_gb300 import sif
    L = sif.load()
    assert L.sif_probe_reciprocal(None, None, -1, None) == sif.EINVAL
    assert L.sif_probe_reciprocal(None, None, 4, None) == sif.EINVAL
    assert L.sif_probe_reciprocal(None, None, 0, None) == sif.OK
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    assert sif.probe_reciprocal(e).numel() == 0
