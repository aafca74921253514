"""Properties that fix Keys' cubic convolution kernel with a = -1/2, checked on
any implementation of it (the oracle's ``keys_cubic``, the brute-force form's
``_keys``, or a planted mistake).

Each check comes from the mathematics of the kernel, not from its formula:

* interpolation: k(0) = 1 and k(n) = 0 at the other integers, support |s| < 2;
* even symmetry;
* partition of unity: sum_i k(f - i) = 1 for every f;
* reproduction of linear and quadratic sequences: sum_i i^d k(f - i) = f^d
  for d = 1, 2 (a = -1/2 is the member of Keys' family with third-order
  accuracy; every other a already fails d = 1);
* continuity of the value and of the first derivative at |s| = 0, 1 and 2
  (one-sided difference quotients on both sides agree);
* the midpoint weights of the Catmull-Rom spline, -1/16, 9/16, 9/16, -1/16
  (the cubic Hermite interpolant with central-difference tangents, built
  from the Hermite basis in ``catmull_rom``), and agreement with that spline
  at arbitrary fractions.
"""
import numpy as np

F_GRID = np.linspace(0.0, 1.0, 41)[:-1]


def catmull_rom(p0, p1, p2, p3, f):
    """Cubic Hermite interpolant between p1 (f = 0) and p2 (f = 1) with the
    tangents (p2 - p0) / 2 and (p3 - p1) / 2, from the Hermite basis
    h00 = 2f^3 - 3f^2 + 1, h10 = f^3 - 2f^2 + f, h01 = -2f^3 + 3f^2,
    h11 = f^3 - f^2."""
    h00 = 2 * f ** 3 - 3 * f ** 2 + 1
    h10 = f ** 3 - 2 * f ** 2 + f
    h01 = -2 * f ** 3 + 3 * f ** 2
    h11 = f ** 3 - f ** 2
    return h00 * p1 + h10 * (p2 - p0) / 2 + h01 * p2 + h11 * (p3 - p1) / 2


def keys_failures(k):
    """List of the properties above that the scalar-or-array kernel ``k``
    violates (empty for a correct kernel)."""
    kv = lambda s: np.asarray(k(np.asarray(s, dtype=np.float64)), dtype=np.float64)  # noqa: E731
    bad = []
    ints = np.arange(-4, 5, dtype=np.float64)
    if np.abs(kv(ints) - (ints == 0)).max() > 1e-15:
        bad.append("interpolating")
    s = np.linspace(-3.0, 3.0, 601)
    if np.abs(kv(s) - kv(-s)).max() > 1e-15:
        bad.append("even")
    if np.abs(kv(s[np.abs(s) >= 2.0])).max() > 0.0:
        bad.append("support")
    taps = range(-2, 4)
    for d, name in ((0, "partition of unity"), (1, "linear reproduction"), (2, "quadratic reproduction")):
        tot = sum(float(i) ** d * kv(F_GRID - i) for i in taps)
        if np.abs(tot - F_GRID ** d).max() > 1e-12:
            bad.append(name)
    h = 1e-6
    for s0 in (0.0, 1.0, 2.0):
        left = (kv(s0) - kv(s0 - h)) / h
        right = (kv(s0 + h) - kv(s0)) / h
        if abs(float(kv(s0 - 1e-12) - kv(s0 + 1e-12))) > 1e-9:
            bad.append(f"continuous at {s0}")
        if abs(float(left - right)) > 1e-4:
            bad.append(f"C1 at {s0}")
    mid = kv(np.array([1.5, 0.5, -0.5, -1.5]))
    if np.abs(mid - np.array([-1, 9, 9, -1]) / 16.0).max() > 1e-15:
        bad.append("Catmull-Rom midpoint weights")
    rng = np.random.default_rng(7)
    p = rng.standard_normal((4, 50))
    f = rng.uniform(0.0, 1.0, 50)
    got = p[0] * kv(f + 1) + p[1] * kv(f) + p[2] * kv(1 - f) + p[3] * kv(2 - f)
    if np.abs(got - catmull_rom(p[0], p[1], p[2], p[3], f)).max() > 1e-12:
        bad.append("Catmull-Rom spline")
    return bad
