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


@pytest.mark.parametrize("use_graph", [True, False])
def test_mode_records_match_oracle(ora, use_graph):
    """lb_batch_record_modes: the six transverse velocity modes each step
    records, per replica, against oracle.transverse_modes of the state that
    step collides (uneven boxes, gammas, noise, a recording started after two
    unrecorded steps, steps past the capacity dropped); lb_batch_mode_acf
    against oracle.mode_autocorrelation of the same records."""
    shapes = [(8, 8, 8), (12, 10, 8), (6, 5, 7), (16, 16, 16)]
    n, cap, nsteps = len(shapes), 12, 14
    stream = torch.cuda.Stream()
    B = L.Batch(shapes, seeds=[21 + k for k in range(n)], replicas=list(range(n)), kT=1e-4, stream=stream, **GAM)
    us = [inputs.shear_wave(s, 0.01) + inputs.gaussian_field(s, 3, 1e-3, seed=30 + k) for k, s in enumerate(shapes)]
    rec = torch.full((n, cap, 12), float("nan"), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for k in range(n):
            L.lb_batch_init_equilibrium(B.b, k, None, _dev(us[k]))
        L.lb_batch_step(B.b, 2, use_graph)
        L.lb_batch_record_modes(B.b, rec, cap)
        L.lb_batch_step(B.b, 5, use_graph)
        L.lb_batch_step(B.b, nsteps - 5, use_graph)
    L.lb_batch_sync(B.b)
    got = rec.cpu().numpy()
    for k, s in enumerate(shapes):
        p = ora.make_params(s, kT=1e-4, seed=21 + k, replica=k, **GAM)
        pops = ora.run(p, ora.equilibrium(p, None, us[k]), 2)
        want = np.zeros((cap, 6), dtype=np.complex128)
        for t in range(cap):
            want[t] = ora.transverse_modes(p, pops)
            pops = ora.step(p, pops, None, 2 + t)
        V = float(np.prod(s))
        g = (got[k, :, 0::2] + 1j * got[k, :, 1::2]) / V
        check("mode records replica %d %s" % (k, s), np.stack([g.real, g.imag]), np.stack([want.real, want.imag]),
              1e-5, 1e-5)
    acf = torch.empty((n, 6), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        L.lb_batch_mode_acf(B.b, rec, cap, 1, cap, 5, acf)
    stream.synchronize()
    for k, s in enumerate(shapes):
        V = float(np.prod(s))
        series = (got[k, :, 0::2] + 1j * got[k, :, 1::2]) / V
        want = ora.mode_autocorrelation(series, 1, cap, 5)
        check("mode acf replica %d" % k, acf[k].cpu().numpy(), want, 1e-12, 1e-12)
    with pytest.raises(L.LBError):
        L.lb_batch_mode_acf(B.b, rec, cap, 0, cap + 1, 3, acf)
    B.close()


def test_velocity_autocorrelation_512_replicas(ora):
    """The batched workload as configured: 512 fluctuating replicas (edges
    from {16, 24, 32, 48, 64} drawn with seed 7, replica r keyed by seed r),
    kT = 1e-4, 2000 steps from rest in one graph-captured persistent launch
    that records the transverse modes.  For every edge length, the replicas'
    mean velocity autocorrelation matches the exact linear theory of the
    update (tests/lb_linear.py: variance kT / (rho0 V) once thermalised, decay
    by the shear eigenvalue lambda(L) per step, the transient from rest
    included) within five standard errors of the replica mean."""
    import lb_linear as LL
    edges = inputs.replica_edges(512, 7)
    shapes = [(e, e, e) for e in edges]
    n, T, max_lag, kT = 512, 2000, 200, 1e-4
    stream = torch.cuda.Stream()
    B = L.Batch(shapes, kT=kT, stream=stream)
    rec = torch.empty((n, T, 12), dtype=torch.float64, device="cuda")
    acf = torch.empty((n, max_lag + 1), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        L.lb_batch_init_equilibrium(B.b)
        L.lb_batch_record_modes(B.b, rec, T)
        L.lb_batch_step(B.b, T, True)
        L.lb_batch_mode_acf(B.b, rec, T, 0, T, max_lag, acf)
    assert L.lb_batch_sync(B.b) == (L.LB_OK, 0)
    A = acf.cpu().numpy()
    tables = ora.tables()
    taus = [0, 1, 10, 50, 100, 200]
    ed = np.array(edges)
    for e in sorted(set(edges)):
        sel = A[ed == e][:, taus]
        V = float(e) ** 3
        want = LL.transverse_acf(e, tables, kT, 1.0, V, taus, 0, T)
        mean = sel.mean(0)
        se = sel.std(0, ddof=1) / np.sqrt(sel.shape[0])
        z = (mean - want) / se
        lam = LL.shear_eigenvalue(e, tables).real
        print("L=%d (%d replicas) acf / (kT/rho0 V): %s theory %s z %s lambda %.6f" % (
            e, sel.shape[0], np.round(mean / (kT / V), 4), np.round(want / (kT / V), 4), np.round(z, 2), lam))
        assert np.all(np.abs(z) < 5), (e, z)
    B.close()
