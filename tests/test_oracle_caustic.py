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


# ---------------------------------------------------------------- first arrival behind the fold

def _rhs_T(s, u):
    """Ray equations in the analytic lens (dx/ds = p/n, dp/ds = grad n) with dT/ds = n."""
    x, y, px, py, T = u
    e = EPS * math.exp(-(x * x + y * y) / SIGMA ** 2)
    n = N0 * (1 + e)
    return [px / n, py / n, N0 * e * (-2 * x / SIGMA ** 2), N0 * e * (-2 * y / SIGMA ** 2), n]


def _shoot(th, smax=0.2):
    return solve_ivp(_rhs_T, (0.0, smax), [R, 0.0, N0 * math.cos(th), N0 * math.sin(th), 0.0],
                     rtol=1e-11, atol=1e-16, max_step=5e-4, dense_output=True)


def _closest(sol, xn, yn):
    """Signed lateral offset of node (xn, yn) from the ray at its closest approach, and the
    travel time there; None if the ray never passes the node."""
    from scipy.optimize import brentq
    ss = np.linspace(0.0, sol.t[-1], 1000)
    U = sol.sol(ss)
    d = (U[0] - xn) * U[2] + (U[1] - yn) * U[3]
    k = np.where(np.diff(np.sign(d)) != 0)[0]
    if len(k) == 0:
        return None
    foot = lambda s: (lambda u: (u[0] - xn) * u[2] + (u[1] - yn) * u[3])(sol.sol(s))
    s = brentq(foot, ss[k[0]], ss[k[0] + 1], xtol=1e-14)
    u = sol.sol(s)
    return (u[2] * (yn - u[1]) - u[3] * (xn - u[0])) / math.hypot(u[2], u[3]), u[4]


def exact_arrivals(nodes):
    """Every ray from the transducer at (R, 0) that passes through each node (two-point
    shooting on the launch angle, Fermat's principle: each is a stationary path), with its
    travel time. Independent of the oracle: scipy's adaptive Runge-Kutta on the analytic medium."""
    from scipy.optimize import brentq
    ths = math.pi + np.linspace(-0.05, 0.05, 101)
    fam = [_shoot(t) for t in ths]
    out = []
    for xn, yn in nodes:
        h = [_closest(s, xn, yn) for s in fam]
        arr = []
        for k in range(len(ths) - 1):
            if h[k] is None or h[k + 1] is None or h[k][0] * h[k + 1][0] > 0:
                continue
            th = brentq(lambda t: _closest(_shoot(t), xn, yn)[0], ths[k], ths[k + 1], xtol=1e-13)
            arr.append((th, _closest(_shoot(th), xn, yn)[1]))
        out.append(arr)
    return out


def test_first_arrival_behind_the_fold(oracle_mod):
    """Overlapping ray tubes keep the first arrival (reading of the triangulation of Sec. 4.4:
    the smallest interpolated T wins). Behind the caustic of the Gaussian lens each node below
    is reached by three rays of the fan of transducer (R, 0); the table's T there must be the
    earliest of the three exact arrivals, within the oracle's discretisation error (about
    4e-10 s at dx = 0.5 mm), while the later arrivals lie 5-27 ns away. The nodes come in
    mirror pairs about the axis, so a rule that kept the first or the last triangle in ray
    order fails on one of each pair, and one that kept the latest arrival fails everywhere."""
    nodes = [(-0.07, 0.0), (-0.08, 0.0), (-0.075, 0.5e-3), (-0.075, -0.5e-3), (-0.085, 0.5e-3), (-0.085, -0.5e-3)]
    arrivals = exact_arrivals(nodes)
    dx = 0.5e-3
    nx = int(2 * (R + 2 * dx) / dx) + 3
    nx += 1 - nx % 2
    g = P.Geometry(nx=nx, ny=nx, dx=dx, n_xducers=1024, ring_radius=R)
    o = oracle_mod.Oracle(g)
    X, Y = g.coords()
    f6 = o.fields(N0 * (1 + EPS * np.exp(-(X ** 2 + Y ** 2) / SIGMA ** 2)))
    tb = o.tables(f6, fans=np.array([0], np.int32))
    pos = {int(v): k for k, v in enumerate(o.idx)}
    for (xn, yn), arr in zip(nodes, arrivals):
        assert len(arr) == 3, ((xn, yn), arr)             # inside the fold: three arrivals
        Ts = sorted(T for _, T in arr)
        assert Ts[2] - Ts[0] >= 4e-9                      # the latest arrival is well apart
        ix, iy = int(round((xn - g.x0) / dx)), int(round((yn - g.y0) / dx))
        k = pos[iy * nx + ix]
        assert tb.cov[0, k] == 1
        T = tb.T[0, k]
        assert abs(T - Ts[0]) <= 1e-9, ((xn, yn), T, Ts)
        assert abs(T - Ts[2]) >= 3e-9, ((xn, yn), T, Ts)
    # the two off-axis pairs: the earliest arrival comes from opposite sides of the fan
    # (launch angle below pi for +y, above pi for -y), so ray order cannot stand in for T
    first = [min(arr, key=lambda a: a[1])[0] - math.pi for arr in arrivals]
    assert first[2] * first[3] < 0 and first[4] * first[5] < 0
