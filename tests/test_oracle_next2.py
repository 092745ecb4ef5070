"""Pins of the oracle's frequency sets and of the integration on the non-smoothed map
(Sec. 6.3.2: rays traced on the smoothed wavenumber map, travel times and amplitudes
integrated along them on the non-smoothed one; two consecutive frequencies per update).
CPU only."""
import math

import numpy as np
import pytest

from paper_2211_00316_gb300 import phantoms as P

C0 = 1500.0


def ring_geom(N=64, R=45e-3, nx=96, dx=1e-3, **kw):
    return P.Geometry(nx=nx, ny=kw.pop("ny", nx), dx=dx, n_xducers=N, ring_radius=R, **kw)


def xducer(g, e):
    b = 2 * math.pi * e / g.n_xducers
    return np.array([math.cos(b), math.sin(b)]) * g.ring_radius


def test_set_of_one_is_the_single_update(oracle_mod):
    """A set of one frequency is the update of Eq. sound_speed_update (lossless and lossy)."""
    w = P.small_two_disc()
    o = oracle_mod.Oracle(w.geom)
    f, df = 3e5, 1e5
    data, _ = o.predict(f, w.c_true)
    c1, st1, _ = o.update_frequency(f, df, w.c_init, data)
    c2, st2, _ = o.update_set([f], df, w.c_init, data[None])
    np.testing.assert_allclose(c2, c1, rtol=1e-13)
    X, Y = w.geom.coords()
    a0 = 1e-9 * np.exp(-(X ** 2 + Y ** 2) / (2 * 0.02 ** 2))
    data, _ = o.predict_abs(f, w.c_true, a0, 1.4)
    c1, _, _ = o.update_frequency_abs(f, df, w.c_init, a0, 1.4, data)
    c2, _, _ = o.update_set([f], df, w.c_init, data[None], alpha0=a0, y=1.4)
    np.testing.assert_allclose(c2, c1, rtol=1e-13)


def test_two_frequency_peak(oracle_mod):
    """Point scatterer at the ring centre in water (Eqs. preconditioner, sound_speed_update2):
    a set of two frequencies gives the sum of the single-frequency peaks,
    sum_k dA dm0 Delta omega omega_k / (pi c0^2)."""
    g = ring_geom(N=64, nx=97)
    o = oracle_mod.Oracle(g)
    freqs, df = (3e5, 3.1e5), 1e4
    c = np.full((g.ny, g.nx), C0)
    ns, f6 = o.fields_for(c, freqs[0])
    tb = o.tables(f6)
    centre = int(np.flatnonzero(o.idx == (g.ny // 2) * g.nx + g.nx // 2)[0])
    dm0 = 1e-3 / C0 ** 2
    data = []
    for f in freqs:
        w = 2 * math.pi * f
        v = np.zeros(o.X)
        v[centre] = w * w * g.dx ** 2 * dm0
        d = o.direct_green(f, tb.exits)[0] + o.forward(f, tb.T, tb.a, tb.K, v)
        np.fill_diagonal(d, 0)
        data.append(d)
    c_out, st, bad = o.update_set(freqs, df, c, np.stack(data))
    assert bad == 0
    expect = sum(g.dx ** 2 * dm0 * (2 * math.pi * df) * (2 * math.pi * f) / (math.pi * C0 ** 2) for f in freqs)
    k = (g.ny // 2) * g.nx + g.nx // 2
    dm_est = (1.0 / c_out.ravel()[k] ** 2 - 1.0 / C0 ** 2) / g.tau
    assert abs(dm_est / expect - 1) < 1e-8


def _periodic_case(oracle_mod, eps_rel=2e-3):
    """Slowness n0 + eps cos(2 pi ix / w) with w the smoothing window: the window averages every
    full period to zero, so the smoothed map is uniform water and the rays are straight, while
    the non-smoothed map carries the pattern."""
    g = ring_geom(N=64, nx=112)              # x edges farther than w/2 from the ring
    o = oracle_mod.Oracle(g)
    f = 2e5
    w = o.window(f)
    n0 = 1.0 / C0
    ix = np.arange(g.nx)
    prow = eps_rel * n0 * np.cos(2 * math.pi * ix / w)
    c = 1.0 / (n0 + np.broadcast_to(prow, (g.ny, g.nx)))
    return g, o, f, n0, prow, c


def _line_integral_pl(g, prow, pa, pb):
    """Exact integral along the segment pa -> pb of the node values prow[ix] interpolated
    linearly in x (constant in y), and the error bound of the ray's trapezoid rule with
    samples ds apart: ds^2 / 8 times the slope jump along s at every node crossed, plus
    ds^2 / 8 times the largest slope for the final partial step (its increment is the last
    full step's scaled linearly along the chord, Def. ray-parameterisation)."""
    L = float(np.linalg.norm(pb - pa))
    ux = (pb[0] - pa[0]) / L
    xs = g.x0 + g.dx * np.arange(g.nx)
    u0, u1 = (pa[0] - g.x0) / g.dx, (pb[0] - g.x0) / g.dx
    if abs(ux) < 1e-9:
        i = int(math.floor(u0))
        t = u0 - i
        return L * ((1 - t) * prow[i] + t * prow[i + 1]), 1e-16
    lo, hi = min(u0, u1), max(u0, u1)

    def val(u):
        i = min(int(math.floor(u)), g.nx - 2)
        t = u - i
        return (1 - t) * prow[i] + t * prow[i + 1]

    pts = [lo] + [float(k) for k in range(int(math.floor(lo)) + 1, int(math.ceil(hi)))] + [hi]
    integ = sum(0.5 * (val(a) + val(b)) * (b - a) for a, b in zip(pts[:-1], pts[1:])) * g.dx
    kinks = range(int(math.floor(lo)) + 1, int(math.ceil(hi)))
    jump = sum(abs(prow[k + 1] - 2 * prow[k] + prow[k - 1]) for k in kinks) / g.dx
    del xs
    slope = np.abs(np.diff(prow)).max() / g.dx
    return integ / abs(ux), abs(ux) * (jump + slope) * g.ds ** 2 / 8


def test_raw_integration_travel_time(oracle_mod):
    """Sec. 6.3.2: with the non-smoothed map the exit travel time is n0 L plus the line integral
    of the pattern along the (straight) ray, to the trapezoid rule's error; on the smoothed map
    the pattern is absent."""
    g, o, f, n0, prow, c = _periodic_case(oracle_mod)
    ns, f6 = o.fields_for(c, f)
    X, Y = g.coords()
    inner = X ** 2 + Y ** 2 <= (g.ring_radius + 2 * g.dx) ** 2     # every cell a ray touches
    assert np.abs(ns - n0)[inner].max() < 1e-15
    nr = 1.0 / c
    raw = o.tables(f6, fans=[0, 17], nr=nr)
    smooth = o.tables(f6, fans=[0, 17])
    for q, e in enumerate((0, 17)):
        xe = xducer(g, e)
        for j in range(1, g.n_xducers, 5):
            ang = raw.exits[q, j - 1, 0]
            pb = np.array([math.cos(ang), math.sin(ang)]) * g.ring_radius
            L = float(np.linalg.norm(pb - xe))
            integ, tol = _line_integral_pl(g, prow, xe, pb)
            assert abs(raw.exits[q, j - 1, 1] - (n0 * L + integ)) <= tol + 1e-15
            assert abs(smooth.exits[q, j - 1, 1] - n0 * L) <= 1e-15
        assert np.abs(raw.exits[q, :, 1] - smooth.exits[q, :, 1]).max() > 1e3 * 1e-15


def test_raw_integration_amplitude_ratio(oracle_mod):
    """Eq. amplitude-geom-discretised on the non-smoothed map: along a straight ray J = s, so
    a = [ (n(x_1) / n(x)) (ds / s) / ds ]^(1/2) with n the non-smoothed slowness."""
    g, o, f, n0, prow, c = _periodic_case(oracle_mod, eps_rel=2e-2)
    ns, f6 = o.fields_for(c, f)
    e, j = 3, 20
    gam0 = 2 * math.pi * e / g.n_xducers + math.pi / 2 + math.pi * j / g.n_xducers
    xe = xducer(g, e)
    rows = o.trace_ray(xe[0], xe[1], gam0, f6=f6, nr=1.0 / c)

    def n_at(p):
        u = (p[0] - g.x0) / g.dx
        i = int(math.floor(u))
        t = u - i
        return n0 + (1 - t) * prow[i] + t * prow[i + 1]

    n1 = n_at(rows[1, :2])
    for i in range(2, len(rows) - 1, 17):
        s = rows[i, 11]
        ref = math.sqrt(n1 / n_at(rows[i, :2]) / s)
        assert abs(rows[i, 4] / ref - 1) < 1e-9


def test_raw_fixed_point_and_sign(oracle_mod):
    """Data predicted with the non-smoothed integration give no update; a weak slow inclusion
    is recovered with the right sign (Eq. sound_speed_update with the reading of its sign)."""
    g = ring_geom(nx=97)
    o = oracle_mod.Oracle(g)
    X, Y = g.coords()
    ct = C0 - 6.0 * np.exp(-((X - 8e-3) ** 2 + (Y + 5e-3) ** 2) / (2 * (3e-3) ** 2))
    freqs = (2e5, 2.1e5)
    data = np.stack([o.predict_ext(f, ct, raw=True)[0] for f in freqs])
    c_fp, st, bad = o.update_set(freqs, 1e4, ct, data, raw=True)
    assert st[3] <= 1e-24 * np.sum(np.abs(data) ** 2)
    np.testing.assert_allclose(c_fp[g.mask()], ct[g.mask()], rtol=1e-13)
    c_out, st, bad = o.update_set(freqs, 1e4, np.full_like(ct, C0), data, raw=True)
    m = g.mask()
    d_est, d_true = (c_out - C0)[m], (ct - C0)[m]
    assert np.dot(d_est, d_true) / np.linalg.norm(d_est) / np.linalg.norm(d_true) > 0.5
    assert d_est[np.argmin(d_true)] < 0


# --------------------------------------------------------------- ray linking


def _lin_T(c1, g, p, q):
    """Travel time in c = c1 + g y between points p and q (linear-velocity medium, closed form)."""
    cp, cq = c1 + g * p[1], c1 + g * q[1]
    rho2 = (p[0] - q[0]) ** 2 + (p[1] - q[1]) ** 2
    return np.arccosh(1 + g * g * rho2 / (2 * cp * cq)) / abs(g)


def _fan_exits(o, g, e, linear):
    """Exits (angle, T, a, K) of fan e's rays in an analytic medium, traced one by one."""
    N = g.n_xducers
    xe = xducer(g, e)
    out = np.zeros((N - 1, 4))
    for j in range(1, N):
        gam0 = 2 * math.pi * e / N + math.pi / 2 + math.pi * j / N
        rows = o.trace_ray(xe[0], xe[1], gam0, linear=linear)
        L = rows[-1]
        out[j - 1] = (math.atan2(L[1], L[0]), L[2], L[4], L[6])
    return out


def test_linked_rays_meet_the_closed_form_travel_time(oracle_mod):
    """Sec. 4.4 / 6.3.2 ray linking by the secant method: in the linear-velocity medium
    c = c1 + g y (bent rays; the water fan misses the receivers) the linked travel time between
    emitter and receiver equals the arccosh closed form within the integrator's error, and is
    much closer to it than the fan's exit-angle interpolation."""
    g = ring_geom()
    o = oracle_mod.Oracle(g)
    lin = (1500.0, 0.0, 2000.0)
    N = g.n_xducers
    fans = [0, 9, 21, 40]
    exits = np.zeros((N, N - 1, 4))
    for e in fans:
        exits[e] = _fan_exits(o, g, e, lin)
    f = 1e4
    gl, cl, unc, Tl = o.direct_green_linked(f, None, exits, linear=lin)
    assert unc == 0
    gi, _ = o.direct_green(f, exits)
    worst_link, worst_interp = 0.0, 0.0
    for e in fans:
        for r in range(N):
            if r == e or abs(((r - e + N // 2) % N) - N // 2) <= 1:
                continue                           # neighbours: grazing, outside the fan's bracket
            ref = _lin_T(1500.0, 2000.0, xducer(g, e), xducer(g, r))
            worst_link = max(worst_link, abs(Tl[e, r] - ref))
            w = 2 * math.pi * f
            ti = (np.angle(gi[e, r] * np.exp(-1j * (w * ref + math.pi / 4)))) / w   # interpolated T - ref
            worst_interp = max(worst_interp, abs(ti))
    assert worst_link <= 1e-10
    assert worst_interp > 10 * worst_link


def test_linking_in_water_is_the_closed_form(oracle_mod):
    """In water the linked rays are the straight chords: g = App. B's g0 exactly."""
    g = ring_geom()
    o = oracle_mod.Oracle(g)
    ns, f6 = o.fields_for(np.full((g.ny, g.nx), C0), 3e5)
    tb = o.tables(f6)
    f = 3e5
    gl, cl, unc, Tl = o.direct_green_linked(f, f6, tb.exits)
    assert unc == 0
    k = 2 * math.pi * f / C0
    N = g.n_xducers
    for e in range(0, N, 5):
        for r in range(N):
            if r == e:
                continue
            s = np.linalg.norm(xducer(g, e) - xducer(g, r))
            ref = (8 * math.pi * k * s) ** -0.5 * np.exp(1j * (k * s + math.pi / 4))
            assert abs(gl[e, r] - ref) <= 1e-9 * abs(ref)
