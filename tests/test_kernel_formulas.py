"""Host-side checks of closed forms and precision arguments the CUDA kernels
rely on, evaluated in numpy (FP32 where the kernels use FP32) against the
oracle or exact arithmetic.  No GPU is needed.

- The phi_3 / phi_4 stencil weights of the particle kernels (middle weight
  plus C1/C2 for phi_3; the shared square root of phi_4's branches) equal the
  paper's piecewise functions (Eqs. 3point, 4point) as the oracle evaluates
  them.
- The exponential-equilibrium kernel builds exp(lambda.c) - 1 for the 18
  directions from three expm1 values; the product form is exact algebra and
  is accurate to FP32 rounding of its terms (absolute accuracy, which is what
  the population deviations need; where the two components nearly cancel the
  relative accuracy of the small result is lower).
- The sphere kernels decide "inside" in FP32 when the squared distance is
  more than 1e-4 a^2 away from a^2; the FP32 error of that distance is far
  below the margin for centres anywhere in a 1024-node box.
"""
import numpy as np


def _phi3_closed(f):
    up = f >= 0.5
    d = np.where(up, f - 1.0, f)
    w0 = (1.0 + np.sqrt(1.0 - 3.0 * d * d)) / 3.0
    w = np.stack([0.5 * (1.0 - w0 - d), w0, 0.5 * (1.0 - w0 + d)])
    first = np.where(up, 0, -1)
    return first, w


def _phi4_closed(f):
    S = np.sqrt(1.0 + 4.0 * f * (1.0 - f))
    a, b = 3.0 - 2.0 * f, 1.0 + 2.0 * f
    return -1, np.stack([(a - S) / 8, (a + S) / 8, (b + S) / 8, (b - S) / 8])


def test_phi3_phi4_closed_forms_equal_the_paper(ora):
    for f in np.linspace(0.0, 1.0, 1001, endpoint=False):
        first, w = _phi3_closed(np.array(f))
        want = [ora.phi(3, (int(first) + k) - f) for k in range(3)]
        assert np.allclose(w, want, rtol=0, atol=1e-14), f
        first, w = _phi4_closed(np.array(f))
        want = [ora.phi(4, (first + k) - f) for k in range(4)]
        assert np.allclose(w, want, rtol=0, atol=1e-14), f


def test_direction_exponentials_from_three_expm1():
    rng = np.random.default_rng(0)
    dirs = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0), (1, -1, 0),
            (-1, 1, 0), (-1, -1, 0), (0, 1, 1), (0, 1, -1), (0, -1, 1), (0, -1, -1), (1, 0, 1), (-1, 0, 1),
            (1, 0, -1), (-1, 0, -1)]
    worst = 0.0
    for _ in range(200):
        lam = rng.uniform(-0.5, 0.5, 3).astype(np.float32)
        ep = np.expm1(lam).astype(np.float32)
        em = (-ep / (np.float32(1) + ep)).astype(np.float32)
        for c in dirs:
            x, scale = np.float32(0), 0.0
            for d in range(3):
                if c[d]:
                    e = ep[d] if c[d] > 0 else em[d]
                    scale += abs(float(e)) + abs(float(x) * float(e))
                    x = np.float32(x + e + x * e)
            exact = np.expm1(np.dot(np.asarray(c, dtype=np.float64), lam.astype(np.float64)))
            worst = max(worst, abs(float(x) - exact) / scale)
    # a few FP32 ulps of the terms: the absolute accuracy the deviations
    # a_i (delta rho + rho (x_i - s) / (1 + s)) need
    assert worst < 5e-7, worst


def test_fp32_inside_margin_covers_the_rounding():
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(2000):
        a = rng.uniform(1.0, 20.0)
        c = rng.uniform(0.0, 1024.0, 3)
        base = np.floor(c - a) - 2
        cf = (c - base).astype(np.float32)
        B = int(np.ceil(2 * a)) + 6
        o = rng.integers(0, B, (64, 3))
        d32 = (o.astype(np.float32) - cf).astype(np.float32)
        d2f = (d32 * d32).sum(1, dtype=np.float32)
        d64 = (base + o) - c
        d2 = (d64 * d64).sum(1)
        worst = max(worst, float(np.abs(d2f - d2).max() / (a * a)))
    assert worst < 1e-5, worst  # ten times below the 1e-4 a^2 margin
