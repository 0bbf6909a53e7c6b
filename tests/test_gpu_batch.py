"""Batched replicas in one persistent, graph-captured launch: parity of every
replica with the FP64 oracle and with the single-box library path, the
autotuner, the bounded grid barrier's timeout path, and the replica-size
workload drawn with seed 7."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0803_2826_gb300 import inputs  # noqa: E402
from paper_0803_2826_gb300 import lbfluct as L  # noqa: E402
from parity_util import check  # noqa: E402

GAM = dict(gamma_shear=0.2, gamma_bulk=-0.3, gamma_odd=0.4, gamma_even=-0.1)
SHAPES = [(6, 5, 7), (8, 8, 8), (4, 9, 5), (16, 16, 16), (12, 10, 14), (33, 3, 2)]


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_matches_oracle_and_single_box(ora, use_graph):
    c, a, e, w, opp = ora.tables()
    aa = a[:, None, None, None]
    stream = torch.cuda.Stream()
    B = L.Batch(SHAPES, seeds=[11 + k for k in range(len(SHAPES))], replicas=list(range(len(SHAPES))),
                kT=1e-4, stream=stream, **GAM)
    us = [inputs.shear_wave(s, 0.01) + inputs.gaussian_field(s, 3, 1e-3, seed=k) for k, s in enumerate(SHAPES)]
    with torch.cuda.stream(stream):
        for k, s in enumerate(SHAPES):
            L.lb_batch_init_equilibrium(B.b, k, None, _dev(us[k]))
        L.lb_batch_step(B.b, 4, use_graph)
        L.lb_batch_step(B.b, 3, use_graph)
    L.lb_batch_sync(B.b)
    assert L.lb_batch_get_step(B.b) == 7
    for k, s in enumerate(SHAPES):
        got = B.get_populations(k).cpu().numpy()
        p = ora.make_params(s, kT=1e-4, seed=11 + k, replica=k, **GAM)
        want = ora.run(p, ora.equilibrium(p, None, us[k]), 7)
        check("batch replica %d %s vs oracle" % (k, s), got - aa, want - aa, 5e-6, 2e-5)
        lat = L.Lattice(s, kT=1e-4, seed=11 + k, replica=k, **GAM)
        lat.init_equilibrium(None, _dev(us[k]))
        lat.step(7)
        single = lat.get_populations().cpu().numpy()
        check("batch replica %d %s vs single box" % (k, s), got - aa, single - aa, 1e-6, 2e-6)
    B.close()


def test_autotune_and_continue(ora):
    shapes = [(16, 16, 16), (24, 24, 24), (32, 32, 32), (16, 16, 16)]
    stream = torch.cuda.Stream()
    B = L.Batch(shapes, kT=1e-4, stream=stream)
    with torch.cuda.stream(stream):
        L.lb_batch_init_equilibrium(B.b)
    cfg, ms = L.lb_batch_autotune(B.b, 1)
    assert cfg.threads in (128, 256, 512) and cfg.grid > 0 and ms > 0
    steps = L.lb_batch_get_step(B.b)
    assert steps > 0  # trial steps advanced the state
    with torch.cuda.stream(stream):
        L.lb_batch_step(B.b, 5, True)
    L.lb_batch_sync(B.b)
    # replica 2 equals a single box advanced the same number of steps
    lat = L.Lattice(shapes[2], kT=1e-4, seed=2, replica=2)
    lat.init_equilibrium()
    lat.step(steps + 5)
    c, a, e, w, opp = ora.tables()
    aa = a[:, None, None, None]
    got = B.get_populations(2).cpu().numpy()
    check("autotuned batch vs single box", got - aa, lat.get_populations().cpu().numpy() - aa, 1e-6, 2e-6)
    B.close()


def test_barrier_timeout_is_reported_and_recoverable():
    """A barrier poll limit of 0 makes every block that is not the last to
    arrive give up at once: the run stops, lb_batch_sync reports LB_ETIMEOUT,
    and after resetting the limit and the state the batch runs again."""
    shapes = [(32, 32, 32)] * 8
    stream = torch.cuda.Stream()
    B = L.Batch(shapes, kT=1e-4, stream=stream)
    L.lb_batch_set_config(B.b, 128, 512, 2)
    assert L.lb_batch_get_config(B.b).grid > 1
    with torch.cuda.stream(stream):
        L.lb_batch_init_equilibrium(B.b)
    L.lb_batch_set_barrier_limit(B.b, 0)
    with torch.cuda.stream(stream):
        L.lb_batch_step(B.b, 3, False)
    st, bits = L.lb_batch_sync(B.b, raise_on_error=False)
    assert st == L.LB_ETIMEOUT and bits & L.LB_DERR_BARRIER
    L.lb_batch_set_barrier_limit(B.b, 1 << 22)
    with torch.cuda.stream(stream):
        L.lb_batch_init_equilibrium(B.b)
        L.lb_batch_step(B.b, 3, True)
    assert L.lb_batch_sync(B.b) == (L.LB_OK, 0)
    B.close()


def test_seed7_replica_workload_subset(ora):
    """The 512-replica workload (edges drawn from {16,24,32,48,64} with seed 7,
    replica r keyed by seed r): 10 steps of the whole batch; mass conserved in
    every replica; replica 0 and the first replica of each size equal single
    boxes."""
    edges = inputs.replica_edges(512, 7)
    shapes = [(L_, L_, L_) for L_ in edges]
    stream = torch.cuda.Stream()
    B = L.Batch(shapes, kT=1e-4, stream=stream)
    with torch.cuda.stream(stream):
        L.lb_batch_init_equilibrium(B.b)
        L.lb_batch_step(B.b, 10, True)
    L.lb_batch_sync(B.b)
    c, a, e, w, opp = ora.tables()
    aa = a[:, None, None, None]
    firsts = sorted({edges.index(v) for v in set(edges)} | {0})
    for r in firsts:
        lat = L.Lattice(shapes[r], kT=1e-4, seed=r, replica=r)
        lat.init_equilibrium()
        lat.step(10)
        got = B.get_populations(r).cpu().numpy()
        check("seed-7 batch replica %d vs single box" % r, got - aa, lat.get_populations().cpu().numpy() - aa,
              1e-6, 2e-6)
        lat.close()
    sums = torch.empty(L.LB_NSUMS, dtype=torch.float64, device="cuda")
    for r in range(0, 512, 37):
        L.lb_batch_moments(B.b, r, None, None, None, sums)
        torch.cuda.synchronize()
        assert abs(sums[0].item()) < 1e-6 * np.prod(shapes[r])
    B.close()
