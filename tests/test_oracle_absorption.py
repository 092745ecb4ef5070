"""Pins of the oracle's lossy, dispersive medium (Sec. 2.2: Eqs. szabo_dispersion_equation,
wave-number, absorption, amplitude-abs-discretised, scattering-potential and the derivative of
|kbar| in Sec. 3.3). CPU only.

Like the lossless pins they compare with what the mathematics fixes: the lossless special case,
closed forms in a uniform lossy medium, scipy's Hankel function at a complex wavenumber, the
adjoint identity, and the closed-form ratio of the preconditioned peak.
"""
import math

import numpy as np
import pytest
from scipy import special

from paper_2211_00316_gb300 import phantoms as P

C0 = 1500.0
Y = 1.4


def alpha0_from_db(db_per_cm_mhz_y, y=Y):
    """alpha0 in Np (rad/s)^-y m^-1 from dB cm^-1 MHz^-y (alpha = alpha0 omega^y)."""
    np_per_m = db_per_cm_mhz_y * 100.0 / (20.0 * math.log10(math.e))
    return np_per_m / (2 * math.pi * 1e6) ** y


def ring_geom(N=64, R=45e-3, nx=96, dx=1e-3, **kw):
    return P.Geometry(nx=nx, ny=kw.pop("ny", nx), dx=dx, n_xducers=N, ring_radius=R, **kw)


def xducer(g, e):
    b = 2 * math.pi * e / g.n_xducers
    return np.array([math.cos(b), math.sin(b)]) * g.ring_radius


def wavenumbers(f, a0, y=Y, c=C0):
    """(real k, alpha, complex k~) of Eq. szabo_dispersion_equation."""
    w = 2 * math.pi * f
    al = a0 * w ** y
    k = w / c + al * math.tan(math.pi * y / 2)
    return k, al, k + 1j * al


def test_lossless_special_case(oracle_mod):
    """alpha0 = 0 reduces every lossy entry point to the lossless one."""
    w = P.small_two_disc()
    o = oracle_mod.Oracle(w.geom)
    f = 3e5
    z = np.zeros_like(w.c_true)
    d0, _ = o.predict(f, w.c_true)
    d1, _ = o.predict_abs(f, w.c_true, z, Y)
    np.testing.assert_allclose(d1, d0, rtol=1e-13, atol=1e-13 * np.abs(d0).max())
    c0, _, _ = o.update_frequency(f, 1e5, w.c_init, d0)
    c1, _, _ = o.update_frequency_abs(f, 1e5, w.c_init, z, Y, d0)
    np.testing.assert_allclose(c1, c0, rtol=1e-13)


def test_uniform_lossy_tables(oracle_mod):
    """Uniform c and alpha0: rays are straight, T = n_e s with n_e = k/omega (Eq. wave-number)
    and a = s^-1/2 exp(-alpha s) (Eqs. absorption, App. B), within the error of linear
    interpolation over ray-tube triangles (as for water, plus the absorption factor)."""
    g = ring_geom()
    o = oracle_mod.Oracle(g)
    f = 3e5
    a0 = alpha0_from_db(0.75)
    c = np.full((g.ny, g.nx), C0)
    ns, f6, al = o.fields_for_abs(c, np.full_like(c, a0), Y, f)
    tb = o.tables(f6, al=al)
    assert tb.uncovered == 0 and tb.bad_rays == 0
    k, alpha, _ = wavenumbers(f, a0)
    ne = k / (2 * math.pi * f)
    assert alpha * g.ring_radius > 0.05                       # the absorption is visible
    X, Yc = g.coords()
    xy = np.stack([X.ravel()[o.idx], Yc.ravel()[o.idx]], 1)
    dpsi = math.pi / g.n_xducers
    for e in range(0, g.n_xducers, 3):
        s = np.linalg.norm(xy - xducer(g, e), axis=1)
        tolT = s * dpsi ** 2 / 8 * ne * 1.01 + 1e-15
        assert np.all(np.abs(tb.T[e] - ne * s) <= tolT)
        sm = s - g.ds
        fpp = (1 / (2 * sm) + alpha) ** 2 + 1 / (2 * sm ** 2)   # f''/f of f = s^-1/2 e^-alpha s
        tola = g.ds ** 2 / 8 * fpp + dpsi ** 2 / 4 + alpha * s * dpsi ** 2 / 8
        assert np.all(np.abs(tb.a[e] * np.sqrt(s) * np.exp(alpha * s) - 1) <= tola)
        assert np.all(tb.K[e] == 0)


@pytest.mark.parametrize("db", [0.5, 1.0])
def test_lossy_direct_green_vs_hankel(oracle_mod, db):
    """The exact Green's function of the lossy Helmholtz equation (Eq. greens-wave-equation)
    in a uniform medium is (i/4) H0^(1)(k~ s) (scipy, complex argument). The ray form differs
    by the far-field remainder |.|/(8|k~| s) and by the reference amplitude, which uses the
    water wavenumber k0 (Eq. attenuation_geom_reference): |sqrt(k~/k0) - 1|."""
    g = ring_geom()
    o = oracle_mod.Oracle(g)
    a0 = alpha0_from_db(db)
    c = np.full((g.ny, g.nx), C0)
    N = g.n_xducers
    for f in (2e5, 4e5):
        ns, f6, al = o.fields_for_abs(c, np.full_like(c, a0), Y, f)
        tb = o.tables(f6, al=al)
        gd, _ = o.direct_green(f, tb.exits)
        k, alpha, kt = wavenumbers(f, a0)
        k0 = 2 * math.pi * f / C0
        ref = abs(np.sqrt(kt / k0) - 1)
        for e in range(0, N, 7):
            for r in range(N):
                if r == e:
                    continue
                s = np.linalg.norm(xducer(g, e) - xducer(g, r))
                exact = 0.25j * special.hankel1(0, kt * s)
                tol = abs(gd[e, r]) * (1.01 / (8 * abs(kt) * s) + 1.01 * ref) + 1e-15
                assert abs(gd[e, r] - exact) <= tol


def test_lossy_adjoint_identity(oracle_mod):
    """<F dm, R> = <dm, F* R> with the complex scattering potential Upsilon_m = omega c k~
    (Eq. scattering-potential) on a heterogeneous lossy medium, to 1e-12."""
    w = P.small_two_disc()
    g = w.geom
    o = oracle_mod.Oracle(g)
    f = 3e5
    X, Yc = g.coords()
    a0 = alpha0_from_db(1.0) * np.exp(-(X ** 2 + Yc ** 2) / (2 * 0.02 ** 2))
    ns, f6, al = o.fields_for_abs(w.c_true, a0, Y, f)
    tb = o.tables(f6, al=al)
    ups = o.upsilon(f, w.c_true.ravel()[o.idx], a0.ravel()[o.idx], Y)
    assert np.abs(ups.imag).max() > 1e-3 * np.abs(ups.real).max()
    rng = np.random.default_rng(2)
    dm = rng.standard_normal(o.X) * 1e-9
    R = rng.standard_normal((o.N, o.N)) + 1j * rng.standard_normal((o.N, o.N))
    D = o.forward_c(f, tb.T, tb.a, tb.K, ups * g.dx ** 2 * dm)
    lhs = np.vdot(D, R)
    rhs = np.dot(dm, o.adjoint_plain_c(f, tb.T, tb.a, tb.K, ups, R))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_lossy_backprojection_peak_ratio(oracle_mod):
    """Point scatterer at the centre of a uniform lossy medium (Eqs. sound_speed_update2,
    scattering-potential, derivative of |kbar|): the reciprocal Green's functions cancel the
    Green's functions exactly, so the preconditioned peak is the lossless one times
    |kbar||d|kbar|/d omega| / Upsilon_m * Upsilon_m over its lossless value:
    (k / k0) (1 + c0 y tan(pi y/2) omega^(y-1) alpha0)."""
    g = ring_geom(N=64, nx=97)
    o = oracle_mod.Oracle(g)
    f, df = 3e5, 1e5
    c = np.full((g.ny, g.nx), C0)
    a0 = alpha0_from_db(1.0)
    A0 = np.full_like(c, a0)
    ns, f6, al = o.fields_for_abs(c, A0, Y, f)
    tb = o.tables(f6, al=al)
    centre = int(np.flatnonzero(o.idx == (g.ny // 2) * g.nx + g.nx // 2)[0])
    dm0 = 1e-3 / C0 ** 2
    w = 2 * math.pi * f
    v = np.zeros(o.X, np.complex128)
    v[centre] = o.upsilon(f, C0, a0, Y) * g.dx ** 2 * dm0
    gd, _ = o.direct_green(f, tb.exits)
    data = gd + o.forward_c(f, tb.T, tb.a, tb.K, v)
    for e in range(g.n_xducers):
        data[e, e] = 0
    c_out, st, bad = o.update_frequency_abs(f, df, c, A0, Y, data)
    assert bad == 0
    k, alpha, kt = wavenumbers(f, a0)
    lossless = g.dx ** 2 * dm0 * (2 * math.pi * df) * w / (math.pi * C0 ** 2)
    ratio = (k / (w / C0)) * (1 + C0 * Y * math.tan(math.pi * Y / 2) * w ** (Y - 1) * a0)
    assert abs(ratio - 1) > 1e-4                               # the lossy factor is visible
    kk = (g.ny // 2) * g.nx + g.nx // 2
    dm_est = (1.0 / c_out.ravel()[kk] ** 2 - 1.0 / C0 ** 2) / g.tau
    assert abs(dm_est / (lossless * ratio) - 1) < 1e-8


def test_lossy_fixed_point_and_sign(oracle_mod):
    """Data predicted on the current lossy model give no update (Eq. residual); a weak slow
    inclusion inside an absorbing region is recovered with the right sign."""
    g = ring_geom(nx=97)
    o = oracle_mod.Oracle(g)
    X, Yc = g.coords()
    A0 = alpha0_from_db(0.8) * (X ** 2 + Yc ** 2 <= (0.02) ** 2)
    ct = C0 - 6.0 * np.exp(-((X - 8e-3) ** 2 + (Yc + 5e-3) ** 2) / (2 * (3e-3) ** 2))
    f = 2e5
    data, _ = o.predict_abs(f, ct, A0, Y)
    c_fp, st, bad = o.update_frequency_abs(f, 1e5, ct, A0, Y, data)
    assert st[3] <= 1e-24 * np.sum(np.abs(data) ** 2)
    np.testing.assert_allclose(c_fp[g.mask()], ct[g.mask()], rtol=1e-13)
    c_out, st, bad = o.update_frequency_abs(f, 1e5, np.full_like(ct, C0), A0, Y, data)
    m = g.mask()
    d_est, d_true = (c_out - C0)[m], (ct - C0)[m]
    assert np.dot(d_est, d_true) / np.linalg.norm(d_est) / np.linalg.norm(d_true) > 0.5
    assert d_est[np.argmin(d_true)] < 0
