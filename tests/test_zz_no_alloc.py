"""The allocation-free deflation projection against the allocating one.

smpm_apply_deflation_noalloc() exists for callers that cannot allocate device
memory at the time they call (real-time loops that must not meet the
allocator's latency or synchronisation, host applications that fix the
library's device memory up front): it keeps its coarse scratch in a fixed
device array inside the library.  This test calls it through the C ABI twice in a row (so the second
call runs on scratch left over by the first) and checks each result against
smpm_apply(kind=2) on the same handle, within the tolerance the operator
parity tests use; it also checks the size limit and the device-pointer rule.
The file name sorts last so a stop-at-first-failure run has already run every
other test if this one fails.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smpm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_01756_gb300 import smpm as m
    m.load()
    return m


def _rel(a, b):
    return max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)),
               float((a - b).abs().max() / b.abs().max()))


@pytest.mark.parametrize("shape,groups", [((8, 2, 8, 4.0, 1.0), 0), ((8, 2, 8, 4.0, 1.0), 1),
                                          ((40, 3, 7, 10.0, 1.0), 0)])
def test_noalloc_matches_apply_twice(smpm, shape, groups):
    grid = smpm.make_grid(*shape, deflation_groups=groups)
    s = smpm.Solver(grid, 0.0, torch.cuda.current_stream())
    gen = torch.Generator(device="cpu").manual_seed(7)
    for call in range(2):
        nrhs = 3 if call == 0 else 2                      # second call: other size, stale scratch
        x = torch.randn(nrhs, s.k, generator=gen, dtype=torch.float64).cuda()
        y_ref = torch.empty_like(x)
        s.apply("P", x, y_ref)
        y = torch.full_like(x, float("nan"))
        s.apply_deflation_noalloc(x, y)
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
        assert _rel(y, y_ref) < 1e-12, (call, _rel(y, y_ref))
    s.close()


def test_noalloc_largest_accepted_size_and_in_place(smpm):
    """The largest batch that fits the scratch array (2 * nrhs * d just below
    SMPM_NOALLOC_MAX_DOUBLES: the coarse vectors fill it up to its last
    entries), and the in-place form y = x."""
    grid = smpm.make_grid(40, 3, 7, 10.0, 1.0)            # d = 39 coarse unknowns
    s = smpm.Solver(grid, 0.0, torch.cuda.current_stream())
    nrhs = 65536 // (2 * 39)                              # 840: 65520 doubles
    gen = torch.Generator(device="cpu").manual_seed(9)
    x = torch.randn(nrhs, s.k, generator=gen, dtype=torch.float64).cuda()
    y_ref = torch.empty_like(x)
    s.apply("P", x, y_ref)
    y = torch.full_like(x, float("nan"))
    s.apply_deflation_noalloc(x, y)
    torch.cuda.synchronize()
    assert _rel(y, y_ref) < 1e-12
    xi = x[:5].clone()
    s.apply_deflation_noalloc(xi, xi)
    torch.cuda.synchronize()
    assert _rel(xi, y_ref[:5]) < 1e-12
    s.close()


def test_noalloc_rejects_oversize_and_host_buffers(smpm):
    grid = smpm.make_grid(40, 3, 7, 10.0, 1.0)            # d = 39 coarse unknowns
    s = smpm.Solver(grid, 0.0, torch.cuda.current_stream())
    too_many = 65536 // (2 * 39) + 1
    x = torch.zeros(too_many, s.k, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(smpm.SmpmError) as e:
        s.apply_deflation_noalloc(x, y)
    assert e.value.code == smpm.SMPM_EINVAL and "SMPM_NOALLOC_MAX_DOUBLES" in str(e.value)
    xh = np.zeros(s.k)
    yh = np.zeros(s.k)
    with pytest.raises(smpm.SmpmError):
        s.apply_deflation_noalloc(xh, yh)
    s.close()
