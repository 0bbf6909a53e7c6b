"""The index-checking build of the library (LB_DEBUG_BOUNDS=1 selects
liblbfluct_bounds.so, compiled with -DLB_DEBUG_BOUNDS: every population pull
and store and every particle spread index is tested against its array, a
violation sets LB_DERR_BOUNDS and skips the access) runs the hot paths clean:
the paired and single-node stream-collide kernels with walls, the persistent
phi_2 coupling with chains, the per-sub-step phi_3 coupling, FP16 storage and
the batched kernel.  No error bit is set, and every result equals that of the
ordinary build to 1e-5 of the largest entry (same arithmetic; the checks
only add branches, and the impulse atomics may sum in another order).  Each build
runs in a process of its own (the library is loaded once per process).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, %(root)r)
from paper_0803_2826_gb300 import inputs
from paper_0803_2826_gb300 import lbfluct as L

out = {}
def run_box(tag, shape, **kw):
    lat = L.Lattice(shape, **kw)
    u = inputs.shear_wave(shape, 0.01) + inputs.gaussian_field(shape, 3, 1e-3, seed=2)
    if kw.get("walls"):
        u[:, 0] = 0
        u[:, -1] = 0
    lat.init_equilibrium(None, torch.as_tensor(u).cuda())
    lat.step(5)
    st, bits = lat.sync()
    out[tag] = {"bits": int(bits), "pops": lat.get_populations().double().cpu().numpy().ravel().tolist()}

run_box("pair_walls", (30, 8, 6), kT=1e-4, seed=3, walls=True, body_force=(1e-5, 0, 0))
run_box("single_odd", (7, 5, 9), kT=1e-4, seed=3)
run_box("f16", (12, 10, 8), kT=1e-4, seed=3, dtype=L.LB_F16)

for kern in (2, 3):
    shape = (16, 16, 16)
    lat = L.Lattice(shape, kT=1e-4, seed=4)
    lat.init_equilibrium(None, torch.as_tensor(inputs.shear_wave(shape, 0.01)).cuda())
    pos = torch.as_tensor(inputs.random_walk_chains(2, 24, shape, seed=7)).cuda()
    mom = torch.as_tensor(inputs.maxwell_momenta(48, 1.0, 1e-4, seed=8), dtype=torch.float32).cuda()
    parts = L.particles(48, pos, mom, mass0=1.0, gamma0=2.0)
    for t in range(3):
        cp = L.couple_params(n_substeps=10, dt=0.1, seed=11, md_step0=10 * t, chain_len=24, use_wca=True,
                             eps=0.01, sigma=1.0, k_fene=0.3, r0=1.5, kernel=kern, overlap=(t %% 2 == 1))
        L.lb_couple_particles(lat.h, parts, cp)
        lat.step(1)
    st, bits = lat.sync()
    out["coupled_phi%%d" %% kern] = {"bits": int(bits),
                                     "pops": lat.get_populations().double().cpu().numpy().ravel().tolist(),
                                     "mom": mom.double().cpu().numpy().ravel().tolist()}

stream = torch.cuda.Stream()
B = L.Batch([(8, 8, 8), (12, 12, 12), (7, 5, 9)], kT=1e-4, stream=stream)
with torch.cuda.stream(stream):
    L.lb_batch_init_equilibrium(B.b)
    L.lb_batch_step(B.b, 4, True)
st, bits = L.lb_batch_sync(B.b, raise_on_error=False)
out["batch"] = {"bits": int(bits), "pops": B.get_populations(1).cpu().numpy().ravel().tolist()}
B.close()
print("RESULT " + json.dumps(out))
"""


def _run(bounds):
    env = dict(os.environ)
    env["LB_DEBUG_BOUNDS"] = "1" if bounds else "0"
    r = subprocess.run([sys.executable, "-c", SCRIPT % {"root": ROOT}], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_bounds_build_runs_clean_and_matches():
    plain = _run(False)
    checked = _run(True)
    assert os.path.exists(os.path.join(ROOT, "paper_0803_2826_gb300", "liblbfluct_bounds.so"))
    for tag, v in checked.items():
        assert v["bits"] == 0, (tag, hex(v["bits"]))
        assert plain[tag]["bits"] == 0
        for key in v:
            if key == "bits":
                continue
            a, b = np.array(v[key]), np.array(plain[tag][key])
            scale = max(np.abs(b).max(), 1e-30)
            assert np.abs(a - b).max() <= 1e-5 * scale, (tag, key, np.abs(a - b).max() / scale)
