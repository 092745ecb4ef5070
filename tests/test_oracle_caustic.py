"""Pin of the caustic count K (Eq. phase-discretised: K counts the sign changes of the ray
Jacobian J along a ray) in a medium that focuses rays. CPU only.

Medium: a Gaussian slowness lens n = n0 (1 + eps exp(-r^2 / sigma^2)) at the centre of a ring
of radius 100 mm. The central ray from the transducer at (R, 0) passes through the lens; its
neighbours are bent back across it and meet it at the caustic, where J changes sign. Where
that happens is fixed by the ray equations alone (dx/ds = p/n, dp/ds = grad n): here two
neighbouring rays are integrated with scipy's adaptive Runge-Kutta on the analytic medium
and the caustic is where the perturbed ray crosses the axis. The oracle (bilinear fields from
central differences on the grid, Heun steps of dx/2) must find the sign change of J there up
to its own discretisation error, which is second order: it falls about fourfold when dx is
halved.
"""
import math

import numpy as np
from scipy.integrate import solve_ivp

from paper_2211_00316_gb300 import phantoms as P

R = 100e-3
N0 = 1.0 / 1500.0
EPS, SIGMA = 0.04, 4e-3


def exact_caustic():
    """Arc length from the source at which a ray launched at pi - d (d -> 0) crosses the axis."""
    def rhs(s, u):
        x, y, px, py = u
        e = EPS * math.exp(-(x * x + y * y) / SIGMA ** 2)
        n = N0 * (1 + e)
        return [px / n, py / n, N0 * e * (-2 * x / SIGMA ** 2), N0 * e * (-2 * y / SIGMA ** 2)]

    def crossing(s, u):
        return u[1] if s > 0.01 else 1.0

    crossing.terminal, crossing.direction = True, -1
    out = []
    for d in (3e-5, 1e-5):
        th = math.pi - d
        sol = solve_ivp(rhs, (0.0, 0.3), [R, 0.0, N0 * math.cos(th), N0 * math.sin(th)], events=crossing,
                        rtol=1e-11, atol=1e-15, max_step=2e-4)
        out.append(sol.t_events[0][0])
    assert abs(out[0] - out[1]) < 1e-6                 # converged in d (paraxial limit)
    return out[1]


def oracle_caustic(oracle_mod, dx):
    nx = int(2 * (R + 2 * dx) / dx) + 3
    nx += 1 - nx % 2
    g = P.Geometry(nx=nx, ny=nx, dx=dx, n_xducers=64, ring_radius=R)
    o = oracle_mod.Oracle(g)
    X, Y = g.coords()
    f6 = o.fields(N0 * (1 + EPS * np.exp(-(X ** 2 + Y ** 2) / SIGMA ** 2)))
    rows = o.trace_ray(R, 0.0, math.pi, f6=f6)
    s, J, K = rows[:, 11], rows[:, 3], rows[:, 6]
    assert K[0] == 0 and K[-1] == 1                    # one caustic on the way to the ring
    i = int(np.argmax(K > 0))
    assert np.all(K[:i] == 0) and np.all(K[i:] == 1)
    return s[i - 1] + (s[i] - s[i - 1]) * J[i - 1] / (J[i - 1] - J[i])


def test_caustic_of_a_gaussian_lens(oracle_mod):
    sc = exact_caustic()
    assert 0.12 < sc < 0.17                             # behind the lens, before the far side
    e1 = oracle_caustic(oracle_mod, 0.5e-3) - sc
    e2 = oracle_caustic(oracle_mod, 0.25e-3) - sc
    assert abs(e1) <= 1e-3 and abs(e2) <= 0.3e-3
    assert abs(e1) / abs(e2) > 3.0                      # second order in dx
