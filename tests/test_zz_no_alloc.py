"""The allocation-free moment sums (lb_moment_sums_static) agree with the
sums of lb_moments, through the C ABI, on two calls in a row.

lb_moment_sums_static serves callers that cannot allocate device memory (a
host application whose device memory another framework reserved up front, or
a monitoring loop that must not block on an allocation mid-run); it keeps its
reduction scratch in a static device array.  This file is collected last so
that a run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0803_2826_gb300 import inputs  # noqa: E402
from paper_0803_2826_gb300 import lbfluct as L  # noqa: E402


def _sums_both(lat):
    _, _, _, ref = lat.moments(want_rho=False, want_j=False, want_pi=False, want_sums=True)
    cur, _ = L.lb_state_buffers(lat.h)
    out = torch.full((L.LB_NSUMS,), float("nan"), dtype=torch.float64, device="cuda")
    L.lb_moment_sums_static(lat.params, cur, out)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), out.cpu().numpy()


# (70, 50, 40) has 140000 nodes: three 65536-node chunks, the last one
# partial, so the multi-block partials and the cross-block final sum run.
@pytest.mark.parametrize("dtype", [L.LB_F32, L.LB_F16, L.LB_BF16])
@pytest.mark.parametrize("shape,walls", [((40, 33, 27), False), ((16, 12, 10), True), ((70, 50, 40), True)])
def test_static_sums_match_lb_moments(shape, walls, dtype):
    lat = L.Lattice(shape, kT=1e-4, seed=3, walls=walls, dtype=dtype)
    lat.init_equilibrium(None, torch.as_tensor(inputs.shear_wave(shape, 0.01)).cuda())
    lat.step(3)
    ref1, got1 = _sums_both(lat)
    lat.step(2)  # second call on a different state reuses the static scratch
    ref2, got2 = _sums_both(lat)
    n = np.prod(shape)
    for ref, got in ((ref1, got1), (ref2, got2)):
        assert np.all(np.isfinite(got))
        # the two reductions partition the nodes differently (FP32 per-thread
        # partials): compare to 1e-5 of the sum of |terms|, bounded above by
        # sqrt(N sum m^2) for the first moments
        s2 = ref[19:]
        assert np.all(np.abs(got[19:] - s2) <= 1e-5 * s2), (got[19:] - s2)
        assert np.all(np.abs(got[:19] - ref[:19]) <= 1e-5 * np.sqrt(n * s2)), (got[:19] - ref[:19])
    assert not np.array_equal(ref1, ref2)
    lat.close()


def test_static_sums_reject_oversized_box():
    p = L.make_params((1024, 1024, 512))
    big = torch.empty(256, dtype=torch.uint8, device="cuda")
    out = torch.empty(L.LB_NSUMS, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LBError) as ei:
        L.lb_moment_sums_static(p, big, out)
    assert ei.value.status == L.LB_EINVAL and "static scratch limit" in str(ei.value)
