#!/usr/bin/env python3
"""Throughput benchmark of the fluctuating D3Q19 lattice-Boltzmann hot path
with coupled bead-spring chains, on one GB300 per rank.

Workload (one "step" = one LB step of the whole hot path): a 256^3 periodic
box of FP32 populations at kT = 1e-4 (rho0 = 1, all relaxation eigenvalues 0,
so nu = 1/6), coupled to 64 FENE + WCA chains of 256 monomers (friction
Gamma = 20 / mass 1 in MD units, i.e. 2 per LB time), 10 particle sub-steps of
dt = 0.1 LB times (0.01 MD units) per LB step.  Per step: lb_couple_particles
(10 sub-steps: forces, interpolation, OU update, spreading) then lb_step
(fused stream-collide with noise and the spread impulses).

Inputs are synthetic and seeded.  The 2.55 GB of populations are far larger
than L2 (129 MB), so no flush is needed between steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded slab sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SHAPE = (256, 256, 256)
N_CHAINS, CHAIN_LEN = 64, 256
KT = 1e-4
MASS, GAMMA = 1.0, 2.0          # Gamma = 20 m / tau_MD with h_LB = 0.1 tau_MD
DT, NSUB = 0.1, 10              # dt = 0.01 tau_MD
EPS, SIGMA, K_FENE, R0 = 0.01, 1.0, 0.3, 1.5   # epsilon = 0.01 in lattice energy units
# algorithmic bytes per node of the timed stream-collide launch: populations
# read + written, plus the particle impulses when the launch reads them (the
# serial order); with the overlap the impulse nodes are re-updated by a
# separate small launch and the timed launch reads no impulse field
BYTES_PER_NODE = {"serial": 19 * 4 * 2 + 3 * 4, "overlapped": 19 * 4 * 2}
FALLBACK_HBM_GBS = 6800.0
def workload(box: int = SHAPE[0], phi: int = 2) -> str:
    return ("fluctuating D3Q19 %d^3 periodic FP32 kT=1e-4 + 64 FENE/WCA chains x 256 monomers, "
            "10 MD sub-steps per LB step" % box) + ("" if phi == 2 else ", phi_%d interpolation" % phi)
SLAB = (256, 256, 4)            # CPU sample: same x-y extent, 4 planes, one chain


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched / adjoint / reduced-precision measurements")
    ap.add_argument("--e2e-steps", type=int, default=200,
                    help="steps of the end-to-end loop with host copies")
    ap.add_argument("--serial", action="store_true",
                    help="run the coupling before the LB update instead of overlapping the two")
    ap.add_argument("--box", type=int, default=SHAPE[0],
                    help="edge of the coupled box (smaller boxes for profiling runs only)")
    ap.add_argument("--phi", type=int, choices=[2, 3, 4], default=2,
                    help="interpolation function of the coupling (phi_2 is the headline workload)")
    ap.add_argument("--kernel-only", action="store_true",
                    help="time lb_step alone (no particles) on --shape for each --kT and --dtype")
    ap.add_argument("--shape", default="256,256,256")
    ap.add_argument("--kT", default="0,1e-4")
    ap.add_argument("--dtype", default="f32")
    ap.add_argument("--equilibrium", type=int, default=0, choices=[0, 1],
                    help="with --kernel-only: 1 times the exponential equilibrium's collision")
    ap.add_argument("--batch-profile", default="", metavar="R,S,THREADS,TILE,BPS[,REC]",
                    help="profiling: R replicas of the batched form's edge mix, one launch of S steps "
                         "with the given configuration (no autotuning, no graph; REC = 1 records the "
                         "transverse modes), then exit")
    ap.add_argument("--adjoint-form", action="store_true",
                    help="run only the adjoint form (profiling)")
    ap.add_argument("--batched-form", type=int, default=0, metavar="STEPS",
                    help="run only the batched-replica form with this many steps (profiling)")
    ap.add_argument("--sphere-form", type=int, default=0, metavar="STEPS",
                    help="time only the moving-sphere form for STEPS steps (profiling runs)")
    ap.add_argument("--free-particles", type=int, default=0, metavar="N",
                    help="time coupled steps of N free particles (Gamma = 2, phi_2) in --shape between walls "
                         "(--serial: serial order; profiling runs)")
    return ap.parse_args()


def run_kernel_only(args):
    """lb_step alone: one JSON line per (dtype, kT) with ms per launch and the
    algorithmic bandwidth 2 * 19 * element size bytes per node."""
    import torch
    from paper_0803_2826_gb300 import build as B
    from paper_0803_2826_gb300 import lbfluct as L
    B.build()
    torch.cuda.set_device(0)
    shape = tuple(int(v) for v in args.shape.split(","))
    nodes = shape[0] * shape[1] * shape[2]
    peak, src = _peak_hbm()
    dts = {"f32": (L.LB_F32, 4), "f16": (L.LB_F16, 2), "bf16": (L.LB_BF16, 2)}
    stream = torch.cuda.Stream()
    for dname in args.dtype.split(","):
        code, esz = dts[dname]
        for kT in (float(v) for v in args.kT.split(",")):
            with torch.cuda.stream(stream):
                lat = L.Lattice(shape, kT=kT, seed=1, dtype=code, stream=stream, equilibrium=args.equilibrium)
                lat.init_equilibrium()
                lat.step(args.warmup)
            torch.cuda.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            with torch.cuda.stream(stream):
                for a, b in evs:
                    a.record(stream)
                    lat.step(1)
                    b.record(stream)
            torch.cuda.synchronize()
            ms = sorted(a.elapsed_time(b) for a, b in evs)
            med = ms[len(ms) // 2]
            gbs = 2 * 19 * esz * nodes / (med * 1e-3) / 1e9
            print(json.dumps({"kernel": "k_stream_collide_exp" if args.equilibrium else "k_stream_collide",
                              "dtype": dname, "kT": kT, "shape": shape,
                              "ms_median": med, "ms_min": ms[0], "mlups": nodes / (med * 1e-3) / 1e6,
                              "gbs": gbs, "frac": gbs / peak, "peak": peak, "peak_source": src}))
            lat.close()
    return 0


def run_free_particles(args):
    """Coupled steps of N free point particles (uniform between the walls,
    Gamma = 2 per LB time, 10 sub-steps, phi_2) in a --shape box with walls,
    FP32, kT = 1e-4, g = 1e-6: the particle load of the reduced-precision
    workload on a box of the caller's choosing.  One JSON line with the ms per
    coupled step (overlapped order unless --serial)."""
    import torch
    from paper_0803_2826_gb300 import build as B
    from paper_0803_2826_gb300 import inputs
    from paper_0803_2826_gb300 import lbfluct as L
    B.build()
    torch.cuda.set_device(0)
    shape = tuple(int(v) for v in args.shape.split(","))
    n = args.free_particles
    stream = torch.cuda.Stream()
    pos = inputs.uniform_particles(n, shape, seed=1, zrange=(1.0, shape[2] - 2.0))
    mom = inputs.maxwell_momenta(n, MASS, KT, seed=2)
    lat = L.Lattice(shape, kT=KT, seed=3, walls=True, body_force=(1e-6, 0, 0), stream=stream)
    gpos = torch.as_tensor(pos).cuda()
    gmom = torch.as_tensor(mom, dtype=torch.float32).cuda()
    parts = L.particles(n, gpos, gmom, mass0=MASS, gamma0=GAMMA)
    t = [0]

    def coupled(k):
        for _ in range(k):
            cp = L.couple_params(n_substeps=NSUB, dt=DT, seed=5, md_step0=NSUB * t[0], overlap=not args.serial)
            L.lb_couple_particles(lat.h, parts, cp)
            lat.step(1)
            t[0] += 1

    with torch.cuda.stream(stream):
        lat.init_equilibrium()
        coupled(args.warmup)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
        coupled(args.steps)
        b.record(stream)
    torch.cuda.synchronize()
    st, bits = lat.sync()
    print(json.dumps({"form": "free_particles", "shape": shape, "particles": n, "order": "serial" if args.serial
                      else "overlapped", "steps": args.steps, "ms_per_step": a.elapsed_time(b) / max(args.steps, 1),
                      "error_bits": bits}))
    lat.close()
    return 0


def _peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampler for the timed region (SM clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.close()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k]
                          and not r[5 + k].startswith("Not")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (the slowest
    rank's timings); the identity without a process group."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _cpu_sample(seconds_target=12.0, max_steps=None):
    """Time the FP64 oracle on a bounded sample: a 256 x 256 x 4 periodic slab
    (the workload's per-node work) with one chain of 256 monomers, repeated
    until about `seconds_target` seconds of CPU work."""
    import numpy as np
    import oracle as O
    from paper_0803_2826_gb300 import inputs
    O.build()
    p = O.make_params(SLAB, kT=KT, seed=0)
    pops = O.equilibrium(p)
    pos = inputs.random_walk_chains(1, CHAIN_LEN, SLAB[:2] + (256,), seed=0)
    pos[:, 2] = np.mod(pos[:, 2], SLAB[2])
    mom = inputs.maxwell_momenta(CHAIN_LEN, MASS, KT, seed=1)
    md = O.make_md(1, CHAIN_LEN, eps=EPS, sigma=SIGMA, k_fene=K_FENE, r0=R0)
    nodes = SLAB[0] * SLAB[1] * SLAB[2]
    steps, t0 = 0, time.perf_counter()
    while True:
        pos, mom, facc, _ = O.couple(p, pops, pos, mom, MASS, GAMMA, dt=DT, n_substeps=NSUB, seed=2,
                                     md_step0=NSUB * steps, md=md)
        pops = O.step(p, pops, facc, steps)
        steps += 1
        el = time.perf_counter() - t0
        if (max_steps and steps >= max_steps) or (not max_steps and el >= seconds_target):
            break
    return nodes * steps / el / 1e6, steps, el, O.threads()


def run_reference(args):
    world, rank, local = _dist()
    if rank != 0:
        return 0
    # warm-up steps, then K timed steps; each step is one slab sample
    _cpu_sample(max_steps=max(args.warmup, 1))
    mlups, steps, el, cores = _cpu_sample(max_steps=args.steps)
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload(), "sample": "256x256x4 periodic slab + 1 chain of 256 per step"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": "%d steps of a 256x256x4 slab + 1 x 256-monomer chain" % steps},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch
    from paper_0803_2826_gb300 import build as B
    from paper_0803_2826_gb300 import inputs
    from paper_0803_2826_gb300 import lbfluct as L

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    B.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    shape = (args.box,) * 3
    nodes = shape[0] * shape[1] * shape[2]
    npart = N_CHAINS * CHAIN_LEN
    # the particle state and two slots of moment sums live in one device
    # buffer: positions FP64 [n][3], momenta FP32 [n][3], then the two slots
    # of 38 FP64 sums (the end-to-end loop alternates them between steps)
    pos_b, mom_b, sums_b = npart * 3 * 8, npart * 3 * 4, L.LB_NSUMS * 8
    pos_off = 0
    sums_off = (pos_b + mom_b + 255) // 256 * 256
    sstride = (sums_b + 255) // 256 * 256
    io_bytes = sums_off + 2 * sstride
    with torch.cuda.stream(stream):
        lat = L.Lattice(shape, kT=KT, seed=rank, replica=rank, stream=stream)
        lat.init_equilibrium()
        pos0 = inputs.random_walk_chains(N_CHAINS, CHAIN_LEN, shape, seed=rank)
        mom0 = inputs.maxwell_momenta(npart, MASS, KT, seed=1000 + rank)
        dio = torch.zeros(io_bytes, dtype=torch.uint8, device=dev)
        gpos = dio[pos_off:pos_off + pos_b].view(torch.float64).view(npart, 3)
        gmom = dio[pos_off + pos_b:pos_off + pos_b + mom_b].view(torch.float32).view(npart, 3)
        dsums = tuple(dio[sums_off + sstride * q:sums_off + sstride * q + sums_b].view(torch.float64) for q in (0, 1))
        gpos.copy_(torch.as_tensor(pos0))
        gmom.copy_(torch.as_tensor(mom0, dtype=torch.float32))
    torch.cuda.synchronize()
    parts = L.particles(npart, gpos, gmom, mass0=MASS, gamma0=GAMMA)
    cp = L.couple_params(n_substeps=NSUB, dt=DT, seed=7 + rank, chain_len=CHAIN_LEN, use_wca=True,
                         eps=EPS, sigma=SIGMA, k_fene=K_FENE, r0=R0, overlap=not args.serial, kernel=args.phi)
    t_step = [0]

    def one_step(sums=None, ready=None, cdone=None):
        cp.md_step0 = (NSUB * t_step[0]) & 0xffffffff
        if ready is None:
            L.lb_couple_particles(lat.h, parts, cp)
        else:  # the particle state comes and goes on a copy stream
            L.lb_couple_particles_async(lat.h, parts, cp, ready, cdone)
        if sums is None:
            L.lb_step(lat.h, 1)
        else:  # the step also returns the moment sums of the state it started from
            L.lb_step_sums(lat.h, 1, sums)
        t_step[0] += 1

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
    barrier()
    st, bits = lat.sync()
    assert bits == 0, "device error word 0x%x during warm-up" % bits

    K = args.steps
    # the library's kernel timers: CUDA events around each stream-collide
    # launch and each coupling, on the stream each runs on (with the overlap
    # the coupling runs on the library's own stream)
    L.lb_set_timing(lat.h, K)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = L.lb_get_launch_count(lat.h)
    clocks = Clocks(local)
    barrier()
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        t0.record(stream)
        for k in range(K):
            one_step()
        t1.record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    launches = L.lb_get_launch_count(lat.h) - launches0
    ms_total = t0.elapsed_time(t1)
    sc_sum, sc_n, cp_sum, cp_n = L.lb_get_timing(lat.h)
    assert sc_n == K and cp_n == K, (sc_n, cp_n)
    sc_avg, couple_ms = sc_sum / sc_n, cp_sum / cp_n
    L.lb_set_timing(lat.h, 0)
    st, bits = lat.sync()
    assert bits == 0, "device error word 0x%x" % bits

    # a steadier view of the same loop: max(200, K) steps timed the same way
    # (the JSON line's value stays the K-step measurement)
    KS = max(200, K)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    sissue0 = time.perf_counter()
    with torch.cuda.stream(stream):
        s0.record(stream)
        for _ in range(KS):
            one_step()
        s1.record(stream)
    steady_issue_ms = (time.perf_counter() - sissue0) * 1e3
    barrier()
    steady_ms = s0.elapsed_time(s1)

    # end to end through the public API with host buffers: per step the
    # particle state goes host -> device from pinned memory and the step's
    # result comes back: the particle state (and, in the second loop, also
    # the moment sums, the 38 sums of lb_moments that lb_step_sums accumulates
    # in the step's stream-collide launch).  The copies run on copy streams,
    # pipelined with the compute: the particle state of step k comes back as
    # soon as the coupling of step k has finished (while that step's
    # stream-collide launch still runs) and goes up again as step k+1's input
    # (the host returns the state it received), which only the coupling of
    # step k+1 waits for; the sums of step k come back beside step k+1
    KE = args.e2e_steps
    dpart = dio[pos_off:pos_off + pos_b + mom_b]
    hio = torch.empty(pos_b + mom_b, dtype=torch.uint8, pin_memory=True)
    hio.copy_(dpart.cpu())
    hsums_all = torch.empty((2, L.LB_NSUMS), dtype=torch.float64, pin_memory=True)
    hsums = (hsums_all[0], hsums_all[1])
    cpy, rd = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ready, cdone, done = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()
    rdone = (torch.cuda.Event(), torch.cuda.Event())

    def e2e_loop(with_sums):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        issue0 = time.perf_counter()
        with torch.cuda.stream(stream):
            e0.record(stream)
            cpy.wait_stream(stream)
            rd.wait_stream(stream)
            for k in range(KE):
                with torch.cuda.stream(cpy):
                    if k:
                        cpy.wait_event(cdone)
                        hio.copy_(dpart, non_blocking=True)   # step k-1's particle state
                    dpart.copy_(hio, non_blocking=True)       # step k's input
                    ready.record(cpy)
                if not with_sums:
                    one_step(None, ready, cdone)
                    continue
                if k >= 2:  # the slot's previous sums have reached the host
                    stream.wait_event(rdone[k % 2])
                one_step(dsums[k % 2], ready, cdone)
                done.record(stream)
                with torch.cuda.stream(rd):
                    rd.wait_event(done)
                    hsums[k % 2].copy_(dsums[k % 2], non_blocking=True)
                    rdone[k % 2].record(rd)
            with torch.cuda.stream(cpy):
                cpy.wait_event(cdone)
                hio.copy_(dpart, non_blocking=True)
            stream.wait_stream(cpy)
            stream.wait_stream(rd)
            e1.record(stream)
        issue = (time.perf_counter() - issue0) * 1e3 / KE  # host time to issue a step
        barrier()
        return e0.elapsed_time(e1), issue

    e2e_ms, issue_ms = e2e_loop(False)
    e2e_sums_ms, issue_sums_ms = e2e_loop(True)
    h2d = pos_b + mom_b
    d2h = pos_b + mom_b

    # max over ranks
    ms_total, sc_avg, e2e_ms, e2e_sums_ms, couple_ms, steady_ms = max_over_ranks(
        [ms_total, sc_avg, e2e_ms, e2e_sums_ms, couple_ms, steady_ms], dist, dev)
    if rank != 0:
        dist.destroy_process_group()
        return 0

    ms_per_step = ms_total / K
    value = world * nodes * K / (ms_total * 1e-3) / 1e6
    e2e_value = world * nodes * KE / (e2e_ms * 1e-3) / 1e6
    peak, peak_src = _peak_hbm()
    bpn = BYTES_PER_NODE["serial" if args.serial else "overlapped"]
    achieved = bpn * nodes / (sc_avg * 1e-3) / 1e9
    traffic = _profiled_traffic("serial" if args.serial else "overlapped")
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload(args.box, args.phi), "nodes": nodes, "particles": npart, "substeps": NSUB,
                   "l2": "inputs larger than L2 (2.55 GB populations per replica)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "k_stream_collide",
                     "bytes_per_node": bpn, "ms_per_launch": sc_avg,
                     "coupling_ms_per_step": couple_ms,
                     "coupling": "serial" if args.serial else "overlapped with the stream-collide launch",
                     "peak_source": peak_src},
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": KE, "copies_per_step": {"h2d": 1, "d2h": 1}, "result": "particle state",
                "host_issue_ms_per_step": issue_ms,
                "with_moment_sums": {"value": world * nodes * KE / (e2e_sums_ms * 1e-3) / 1e6, "unit": "MLUPS",
                                     "d2h_bytes_per_step": d2h + sums_b, "copies_per_step": {"h2d": 1, "d2h": 2},
                                     "host_issue_ms_per_step": issue_sums_ms,
                                     "result": "particle state + the 38 moment sums (lb_step_sums)"}},
        "steady": {"steps": KS, "ms_per_step": steady_ms / KS,
                   "value": world * nodes * KS / (steady_ms * 1e-3) / 1e6, "unit": "MLUPS",
                   "host_issue_ms_per_step": steady_issue_ms / KS},
        "clocks": clk,
        "wall_s": wall,
    }
    if world == 1 and not args.no_forms:
        lat.close()
        torch.cuda.empty_cache()
        line["forms"] = _forms(peak)
    if world == 1 and not args.no_cpu_baseline:
        mlups, steps, el, cores = _cpu_sample()
        line["cpu_baseline"] = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                                "sample": "%d steps of a 256x256x4 slab + 1 x 256-monomer chain (%.1f s)"
                                          % (steps, el)}
    print(json.dumps(line))
    if lat.h is not None:
        lat.close()
    if dist:
        dist.destroy_process_group()
    return 0


def _forms(peak):
    """The further forms, each timed with CUDA events against the plain
    FP32 form on the same box:
      batched   512 periodic replicas, edges from {16,24,32,48,64} drawn with
                seed 7, replica r keyed by seed r, kT = 1e-4, FP32: autotuned,
                then 2000 steps in one graph-replayed persistent launch that
                records the transverse velocity modes, and their per-replica
                autocorrelation (see _batched_form);
      adjoint   64^3, kT = 0, force field ~ N(0, 1e-5), kinetic energy of the
                central 16^3 after 500 steps, checkpoints every 50: forward +
                reverse ms per step vs 500 plain FP32 steps;
      interpolation  the headline coupled workload with phi_3 and phi_4;
      spheres   256^3 with 512 moving solid spheres (moving bounce-back);
      exp_equilibrium  256^3 steps with the exponential vs the quadratic equilibrium;
      precision 512^3 between walls, g = 1e-6, kT = 1e-4, 1e5 free point
                particles: ms per coupled LB step with FP16 / BF16 storage vs
                FP32 storage, and the LB step alone."""
    import numpy as np
    import torch
    from paper_0803_2826_gb300 import inputs
    from paper_0803_2826_gb300 import lbfluct as L
    out = {}
    stream = torch.cuda.Stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    # batched replicas
    out["batched"] = _batched_form(stream, peak)

    # adjoint vs plain forward
    out["adjoint"] = _adjoint_form(stream)

    # wider interpolation stencils on the headline workload
    out["interpolation"] = _interpolation_forms(stream)

    # extended particles: moving solid spheres
    out["spheres"] = _sphere_form(stream, peak)

    # the exponential equilibrium against the quadratic one, 256^3 FP32 kT = 1e-4
    exp_eq = {}
    for name, eq in (("quadratic", 0), ("exponential", 1)):
        lat = L.Lattice((256, 256, 256), kT=KT, seed=9, equilibrium=eq, stream=stream)
        with torch.cuda.stream(stream):
            lat.init_equilibrium(None, torch.as_tensor(inputs.shear_wave((256, 256, 256), 0.05)).cuda())
            lat.step(3)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        with torch.cuda.stream(stream):
            a.record(stream)
            lat.step(50)
            b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 50
        exp_eq[name] = {"ms_per_step": ms, "mlups": 256 ** 3 / (ms * 1e-3) / 1e6,
                        "hbm_frac": 152 * 256 ** 3 / (ms * 1e-3) / 1e9 / peak}
        lat.close()
        torch.cuda.empty_cache()
    out["exp_equilibrium"] = exp_eq

    # reduced-precision storage: the configured workload (512^3 between walls,
    # Poiseuille force, 1e5 free point particles with Gamma = 20 in MD units,
    # 10 sub-steps per LB step), and the LB step alone beside it
    shape = (512, 512, 512)
    npart = 100000
    pos = inputs.uniform_particles(npart, shape, seed=1, zrange=(1.0, 510.0))
    mom = inputs.maxwell_momenta(npart, MASS, KT, seed=2)
    prec = {}
    for name, code, esz in (("f32", L.LB_F32, 4), ("f16", L.LB_F16, 2), ("bf16", L.LB_BF16, 2)):
        lat = L.Lattice(shape, dtype=code, kT=KT, seed=3, walls=True, body_force=(1e-6, 0, 0), stream=stream)
        gpos = torch.as_tensor(pos).cuda()
        gmom = torch.as_tensor(mom, dtype=torch.float32).cuda()
        parts = L.particles(npart, gpos, gmom, mass0=MASS, gamma0=GAMMA)
        # serial order: with 1e5 particles in 512^3 the overlapped step's
        # re-update of ~8e5 scattered impulse nodes (19 planes each) costs more
        # than reading the impulse field in the step's own launch
        cpp = L.couple_params(n_substeps=NSUB, dt=DT, seed=5, overlap=False)
        nt = [0]

        def coupled(n):
            for _ in range(n):
                cpp.md_step0 = NSUB * nt[0]
                L.lb_couple_particles(lat.h, parts, cpp)
                lat.step(1)
                nt[0] += 1

        with torch.cuda.stream(stream):
            lat.init_equilibrium()
            coupled(3)
            lat.step(3)
        torch.cuda.synchronize()
        a, b, c = ev(), ev(), ev()
        with torch.cuda.stream(stream):
            a.record(stream)
            coupled(20)
            b.record(stream)
            lat.step(20)
            c.record(stream)
        torch.cuda.synchronize()
        assert lat.sync() == (L.LB_OK, 0)
        ms = a.elapsed_time(b) / 20
        ms_lb = b.elapsed_time(c) / 20
        nfl = 512 * 512 * 510
        prec[name] = {"ms_per_step": ms, "mlups": nfl / (ms * 1e-3) / 1e6,
                      "hbm_frac": 2 * 19 * esz * nfl / (ms * 1e-3) / 1e9 / peak,
                      "lb_only_ms_per_step": ms_lb,
                      "lb_only_hbm_frac": 2 * 19 * esz * nfl / (ms_lb * 1e-3) / 1e9 / peak}
        lat.close()
        del gpos, gmom
        torch.cuda.empty_cache()
        # the same LB step without the noise (kT = 0): what the storage format
        # gives where the arithmetic does not bind
        lat = L.Lattice(shape, dtype=code, kT=0.0, seed=3, walls=True, body_force=(1e-6, 0, 0), stream=stream)
        with torch.cuda.stream(stream):
            lat.init_equilibrium()
            lat.step(3)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            a.record(stream)
            lat.step(20)
            b.record(stream)
        torch.cuda.synchronize()
        assert lat.sync() == (L.LB_OK, 0)
        ms0 = a.elapsed_time(b) / 20
        prec[name]["lb_only_kT0_ms_per_step"] = ms0
        prec[name]["lb_only_kT0_hbm_frac"] = 2 * 19 * esz * nfl / (ms0 * 1e-3) / 1e9 / peak
        lat.close()
        torch.cuda.empty_cache()
    for name in ("f16", "bf16"):
        prec[name]["speedup_vs_f32"] = prec["f32"]["ms_per_step"] / prec[name]["ms_per_step"]
        prec[name]["lb_only_speedup_vs_f32"] = prec["f32"]["lb_only_ms_per_step"] / prec[name]["lb_only_ms_per_step"]
        prec[name]["lb_only_kT0_speedup_vs_f32"] = (prec["f32"]["lb_only_kT0_ms_per_step"]
                                                    / prec[name]["lb_only_kT0_ms_per_step"])
    out["precision"] = {"shape": list(shape), "walls": True, "kT": KT, "particles": npart,
                        "workload": "Poiseuille g = 1e-6 between walls at z = 0, 511, 1e5 free particles "
                                    "(Gamma = 20 MD units), 10 sub-steps per LB step, serial coupling",
                        **prec}
    return out


def _adjoint_form(stream):
    """64^3, kT = 0, force field ~ N(0, 1e-5), kinetic energy of the central
    16^3 after 500 steps, checkpoints every 50: forward + reverse ms per step
    against 500 plain FP32 steps (CUDA events)."""
    import numpy as np
    import torch
    from paper_0803_2826_gb300 import inputs
    from paper_0803_2826_gb300 import lbfluct as L
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    shape, T, K = (64, 64, 64), 500, 50
    f = torch.as_tensor(inputs.gaussian_field(shape, 3, 1e-5, seed=0).astype(np.float32)).cuda()
    lat = L.Lattice(shape, force=f, stream=stream)
    g = torch.empty_like(f)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        lat.init_equilibrium()
        lat.step(20)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    with torch.cuda.stream(stream):
        a.record(stream)
        lat.step(T)
        b.record(stream)
    torch.cuda.synchronize()
    fwd_ms = a.elapsed_time(b) / T
    # one untimed call sizes the handle's reverse-mode arena; the timed calls
    # then allocate nothing (CUDA events on the handle's stream)
    with torch.cuda.stream(stream):
        lat.init_equilibrium()
        L.lb_adjoint_kinetic(lat.h, T, K, (24, 24, 24), (40, 40, 40), g, loss)
    torch.cuda.synchronize()
    a, b, c = ev(), ev(), ev()
    with torch.cuda.stream(stream):
        lat.init_equilibrium()
        a.record(stream)
        L.lb_adjoint_forward(lat.h, T, K, (24, 24, 24), (40, 40, 40), loss)
        b.record(stream)
        L.lb_adjoint_backward(lat.h, g)
        c.record(stream)
    torch.cuda.synchronize()
    fwd_ck_ms = a.elapsed_time(b) / T
    adj_ms = a.elapsed_time(c) / T
    # algorithmic bytes per node and step: forward 152 + 12 (force field);
    # reverse 264 (lambda in and out, the state, the force gradient) plus the
    # recompute of the segment states, 152 + 12
    alg_ratio = (164 + 264 + 164) / 164
    lat.close()
    return {"shape": list(shape), "steps": T, "checkpoint_every": K,
                      "fwd_plus_adj_ms_per_step": adj_ms, "fwd_with_checkpoints_ms_per_step": fwd_ck_ms,
                      "plain_fp32_ms_per_step": fwd_ms, "ratio": adj_ms / fwd_ms,
                      "algorithmic_bytes_ratio": alg_ratio, "loss": loss.item(),
                      "timing": "CUDA events around lb_adjoint_forward + lb_adjoint_backward on the handle's "
                                "stream; the checkpoint arena was allocated by an earlier call"}


def _batched_form(stream, peak, nsteps=2000, max_lag=200, t_begin=1000):
    """512 replicas, autotuned, 2000 steps per graph-replayed persistent
    launch: first without the mode records, then from rest with them
    (lb_batch_record_modes) and their per-replica velocity autocorrelation
    (lb_batch_mode_acf over steps t_begin .. nsteps), summarised per edge
    length as the replicas' mean C(0) / (kT / (rho0 V)) and the mean decay per
    step (C(tau) / C(0))^(1/tau) at tau = 1 and 20 (the shear eigenvalue; the
    hydrodynamic value exp(-nu k^2), nu = 1/6, beside it)."""
    import math

    import numpy as np
    import torch
    from paper_0803_2826_gb300 import inputs
    from paper_0803_2826_gb300 import lbfluct as L
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    edges = inputs.replica_edges(512, 7)
    n = len(edges)
    nodes = int(sum(e ** 3 for e in edges))
    B = L.Batch([(e, e, e) for e in edges], kT=KT, stream=stream)
    rec = torch.empty((n, nsteps, 12), dtype=torch.float64, device="cuda")
    acf = torch.empty((n, max_lag + 1), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        L.lb_batch_init_equilibrium(B.b)
    cfg_plain, _ = L.lb_batch_autotune(B.b, 2)

    def timed():
        a, b = ev(), ev()
        with torch.cuda.stream(stream):
            a.record(stream)
            L.lb_batch_step(B.b, nsteps, True)
            b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    with torch.cuda.stream(stream):
        L.lb_batch_step(B.b, nsteps, True)  # records the graph for this length
    torch.cuda.synchronize()
    ms_plain = timed()
    # the recording kernel, tuned with the records on (its per-tile reduction
    # favours longer tiles); the trial steps' records are dropped by re-arming
    with torch.cuda.stream(stream):
        L.lb_batch_record_modes(B.b, rec, nsteps)
    cfg, _ = L.lb_batch_autotune(B.b, 2)
    with torch.cuda.stream(stream):
        L.lb_batch_step(B.b, nsteps, True)  # graph of the recording kernel
        L.lb_batch_init_equilibrium(B.b)    # rest again; the records restart at the next step
        L.lb_batch_record_modes(B.b, rec, nsteps)
    torch.cuda.synchronize()
    ms_rec = timed()
    with torch.cuda.stream(stream):
        L.lb_batch_mode_acf(B.b, rec, nsteps, t_begin, nsteps, max_lag, acf)
    L.lb_batch_sync(B.b)
    A = acf.cpu().numpy()
    ed = np.array(edges)
    per_edge = {}
    for e in sorted(set(edges)):
        sel = A[ed == e]
        V = float(e) ** 3
        c0 = sel[:, 0].mean()
        per_edge[str(e)] = {
            "replicas": int(sel.shape[0]),
            "c0_over_kT_rho0V": c0 / (KT / V),
            "c0_stderr": sel[:, 0].std(ddof=1) / math.sqrt(sel.shape[0]) / (KT / V),
            "decay_per_step_tau1": sel[:, 1].mean() / c0,
            "decay_per_step_tau20": (sel[:, 20].mean() / c0) ** (1.0 / 20),
            "exp_minus_nu_k2": math.exp(-(1.0 / 6.0) * (2 * math.pi / e) ** 2),
        }
    B.close()
    mk = lambda ms: {"ms": ms, "mlups": nodes * nsteps / (ms * 1e-3) / 1e6,  # noqa: E731
                     "hbm_frac": 152 * nodes * nsteps / (ms * 1e-3) / 1e9 / peak}
    return {"replicas": n, "nodes": nodes, "steps": nsteps, "launches": 1,
            **mk(ms_rec), "plain": mk(ms_plain), "timing": "with the mode records (the configured workload); "
            "'plain' without them",
            "autocorrelation": {"steps": [t_begin, nsteps], "start": "rest", "per_edge": per_edge},
            "config": {"threads": cfg.threads, "tile_nodes": cfg.tile_nodes,
                       "blocks_per_sm": cfg.blocks_per_sm, "grid": cfg.grid},
            "config_plain": {"threads": cfg_plain.threads, "tile_nodes": cfg_plain.tile_nodes,
                             "blocks_per_sm": cfg_plain.blocks_per_sm, "grid": cfg_plain.grid}}


def run_batch_profile(args):
    """One persistent launch of the batched kernel on a smaller replica set,
    in a fixed configuration, timed with CUDA events (the kernel for ncu)."""
    import torch
    from paper_0803_2826_gb300 import build as B
    from paper_0803_2826_gb300 import inputs
    from paper_0803_2826_gb300 import lbfluct as L
    B.build()
    vals = [int(v) for v in args.batch_profile.split(",")]
    r, steps, threads, tile, bps = vals[:5]
    records = len(vals) > 5 and vals[5] != 0
    edges = inputs.replica_edges(r, 7)
    nodes = int(sum(e ** 3 for e in edges))
    stream = torch.cuda.Stream()
    Bt = L.Batch([(e, e, e) for e in edges], kT=KT, stream=stream)
    L.lb_batch_set_config(Bt.b, threads, tile, bps)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rec = torch.empty((len(edges), steps, 12), dtype=torch.float64, device="cuda") if records else None
    with torch.cuda.stream(stream):
        L.lb_batch_init_equilibrium(Bt.b)
        if records:
            L.lb_batch_record_modes(Bt.b, rec, steps)
        a.record(stream)
        L.lb_batch_step(Bt.b, steps, False)
        b.record(stream)
    torch.cuda.synchronize()
    L.lb_batch_sync(Bt.b)
    ms = a.elapsed_time(b)
    peak = _peak_hbm()[0]
    print(json.dumps({"kernel": "k_batch_pair_obs" if records else "k_batch_pair", "replicas": r, "nodes": nodes,
                      "steps": steps,
                      "config": [threads, tile, bps], "ms": ms,
                      "hbm_frac": 152 * nodes * steps / (ms * 1e-3) / 1e9 / peak}))
    Bt.close()
    return 0


def _interpolation_forms(stream, steps=100):
    """The coupled 256^3 workload of the headline line with the three- and
    four-point interpolation functions (27 / 64 stencil nodes per monomer,
    per-sub-step kernels, coupling overlapped with the LB update): ms per
    step and the coupling's ms per step from the library's kernel timers."""
    import torch
    from paper_0803_2826_gb300 import inputs
    from paper_0803_2826_gb300 import lbfluct as L
    npart = N_CHAINS * CHAIN_LEN
    lat = L.Lattice(SHAPE, kT=KT, seed=0, stream=stream)
    with torch.cuda.stream(stream):
        lat.init_equilibrium()
    pos0 = inputs.random_walk_chains(N_CHAINS, CHAIN_LEN, SHAPE, seed=0)
    mom0 = inputs.maxwell_momenta(npart, MASS, KT, seed=1000)
    res = {"steps": steps}
    for phi in (3, 4):
        gpos = torch.as_tensor(pos0).cuda()
        gmom = torch.as_tensor(mom0, dtype=torch.float32).cuda()
        torch.cuda.synchronize()
        parts = L.particles(npart, gpos, gmom, mass0=MASS, gamma0=GAMMA)
        cp = L.couple_params(n_substeps=NSUB, dt=DT, seed=7, chain_len=CHAIN_LEN, use_wca=True, eps=EPS,
                             sigma=SIGMA, k_fene=K_FENE, r0=R0, overlap=True, kernel=phi)

        def run(k, t0):
            for t in range(k):
                cp.md_step0 = NSUB * (t0 + t)
                L.lb_couple_particles(lat.h, parts, cp)
                L.lb_step(lat.h, 1)

        with torch.cuda.stream(stream):
            run(5, 0)
        torch.cuda.synchronize()
        L.lb_set_timing(lat.h, steps)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            run(steps, 5)
            b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        sc_sum, sc_n, cp_sum, cp_n = L.lb_get_timing(lat.h)
        L.lb_set_timing(lat.h, 0)
        st, bits = lat.sync()
        assert bits == 0, "device error word 0x%x (phi_%d)" % (bits, phi)
        nodes = SHAPE[0] * SHAPE[1] * SHAPE[2]
        res["phi%d" % phi] = {"workload": workload(phi=phi), "ms_per_step": ms, "mlups": nodes / (ms * 1e-3) / 1e6,
                              "coupling_ms_per_step": cp_sum / cp_n, "stream_collide_ms": sc_sum / sc_n}
    lat.close()
    torch.cuda.empty_cache()
    return res


def _sphere_form(stream, peak, steps=200):
    """256^3 periodic box, kT = 1e-4, 512 solid spheres of radius 4 (volume
    fraction 0.8 %, neutrally buoyant: m = 4/3 pi a^3 rho0) moving with
    thermal-scale velocities: ms per lb_step_spheres (moving bounce-back,
    sphere update, solid-map motion) against a plain lb_step of the same box;
    algorithmic bytes 152 per node plus the 4-byte solid map."""
    import math
    import numpy as np
    import torch
    from paper_0803_2826_gb300 import inputs
    from paper_0803_2826_gb300 import lbfluct as L
    shape, n, rad = (256, 256, 256), 512, 4.0
    nodes = shape[0] * shape[1] * shape[2]
    lat = L.Lattice(shape, kT=KT, seed=5, stream=stream)
    m0 = 4.0 / 3.0 * math.pi * rad ** 3
    pos = torch.as_tensor(inputs.sphere_centres(n, shape, rad, seed=5)).cuda()
    vel = torch.as_tensor(np.random.default_rng(6).normal(0.0, 0.01, (n, 3))).cuda()
    sph = L.spheres(n, pos, vel, rad, mass0=m0)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    with torch.cuda.stream(stream):
        lat.init_equilibrium()
        lat.step(3)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    with torch.cuda.stream(stream):
        a.record(stream)
        lat.step(steps)
        b.record(stream)
    torch.cuda.synchronize()
    plain = a.elapsed_time(b) / steps
    with torch.cuda.stream(stream):
        L.lb_spheres_place(lat.h, sph)
        for _ in range(5):
            L.lb_step_spheres(lat.h, sph)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    with torch.cuda.stream(stream):
        a.record(stream)
        for _ in range(steps):
            L.lb_step_spheres(lat.h, sph)
        b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    st, bits = lat.sync()
    assert bits == 0, "device error word 0x%x (spheres)" % bits
    lat.close()
    torch.cuda.empty_cache()
    return {"shape": list(shape), "spheres": n, "radius": rad, "steps": steps, "ms_per_step": ms,
            "mlups": nodes / (ms * 1e-3) / 1e6, "hbm_frac": 156 * nodes / (ms * 1e-3) / 1e9 / peak,
            "plain_ms_per_step": plain, "ratio": ms / plain}


def _profiled_traffic(mode):
    """DRAM bytes per stream-collide launch from the committed ncu summary,
    if it was taken on the current source of that kernel, in the same mode
    (serial or overlapped coupling: the launch reads the impulses or not)."""
    path = os.path.join(ROOT, "profiles", "stream_collide_traffic.txt")
    try:
        d = {}
        with open(path) as f:
            for line in f:
                key, sep, val = line.partition(":")
                if sep and key.strip() in ("source_hash", "dram_bytes_per_launch", "mode"):
                    d[key.strip()] = val.strip()
        from paper_0803_2826_gb300 import build as B
        if d.get("source_hash") != B.source_hash(B.STREAM_COLLIDE_FILES) or d.get("mode") != mode:
            return None
        return float(d["dram_bytes_per_launch"])
    except Exception:
        return None


def main():
    args = _args()
    if args.free_particles:
        return run_free_particles(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel_only:
        return run_kernel_only(args)
    if args.batch_profile:
        return run_batch_profile(args)
    if args.adjoint_form:
        import torch
        from paper_0803_2826_gb300 import build as B
        B.build()
        print(json.dumps(_adjoint_form(torch.cuda.Stream())))
        return 0
    if args.batched_form:
        import torch
        n = max(args.batched_form, 44)
        print(json.dumps(_batched_form(torch.cuda.Stream(), _peak_hbm()[0], nsteps=n, t_begin=n // 2,
                                       max_lag=min(200, n // 2 - 1))))
        return 0
    if args.sphere_form:
        import torch
        print(json.dumps(_sphere_form(torch.cuda.Stream(), _peak_hbm()[0], steps=args.sphere_form)))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
