/*
 * rbx_oracle.c -- plain FP64 CPU oracle of the Hessian-free ray-Born update
 * (Javaherian, "Hessian-free ray-Born inversion for quantitative ultrasound
 * tomography of weakly heterogeneous media", arXiv 2211.00316).
 *
 * TEST INFRASTRUCTURE. This file is the independent reference that the CUDA path
 * is checked against. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load it. It shares no code, header, table or constant with the
 * CUDA library. Everything is straightforward loops in double precision, in the
 * order the paper states the steps; OpenMP only spreads independent transducers or
 * grid nodes over threads.
 *
 * Steps (paper section / equation in brackets):
 *   a1  smoothing of the slowness map and its derivatives   [Sec. 4.4, Sec. 6.3.2]
 *   a2  paraxial ray tracing with Heun's method             [Alg. 1; Eqs. ray-equation-reference,
 *                                                             ray-equation-paraxial; Def. ray-parameterisation]
 *   a3  ray-to-grid tables by triangulation                 [Sec. 4.4; Eqs. phase-discretised,
 *                                                             amplitude-geom-discretised]
 *   a4  angular density |d gamma / d e| Delta e              [Eq. sound_speed_update2]
 *   a5  direct Green's function at the receivers            [Eq. 2D_greens; Sec. 6.3]
 *   a6  Green's functions and reciprocal Green's functions  [Eqs. 2D_greens, greens-time-reversed]
 *   a7  ray-Born forward and residual                       [Eqs. perturb1, derivative,
 *                                                             scattering-potential, residual]
 *   a8  preconditioned back-projection (unfactorised sum)  [Eqs. sound_speed_update, sound_speed_update2,
 *                                                             btk-amp-angle]
 *   a9  update of the squared slowness                      [Sec. 3.4, m <- m + tau dm]
 *
 * Absorption and dispersion (Sec. 2.2; the "_abs" entry points): the complex wavenumber
 * k~ = omega/c + alpha (tan(pi y/2) + i), alpha = alpha0 omega^y (Eq. szabo_dispersion_equation).
 * Rays follow the real part k = omega n_e, n_e = 1/c + alpha0 tan(pi y/2) omega^(y-1)
 * (Eqs. wave-number, eikonal), so the phase is omega times the travel time on n_e
 * (Eq. phase-discretised); the amplitude gains A_abs = exp(-int alpha ds) along the ray
 * (Eqs. absorption, amplitude-abs-discretised); the scattering potential is
 * Upsilon_m = omega c k~ (Eq. scattering-potential); the preconditioner's
 * |d|kbar|/d omega| carries the extra term y tan(pi y/2) omega^(y-1) alpha0.
 *
 * Where the paper is silent or ambiguous, the reading taken is stated beside the
 * code below that depends on it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int nx, ny;
    double dx, x0, y0;      /* node (ix,iy) at (x0 + ix dx, y0 + iy dx) */
    int N;                  /* transducers on the ring */
    double R, mask_r, c0, ds;
    int weight_mode;        /* 0 literal scattering angle, 1 isochron */
    double tau;
    const double *beta;     /* angle of transducer e on the ring, counterclockwise order (Sec. 2.1:
                               the elements' positions); NULL: the uniform ring, beta_e = 2 pi e / N */
} og_geom;

/* Position angle beta_e of transducer e: x_e = R (cos beta_e, sin beta_e). */
static double xducer_angle(const og_geom *g, int e) { return g->beta ? g->beta[e] : 2 * M_PI * e / g->N; }

/* Medium seen by the ray tracer. mode 0: bilinear interpolation of six grid fields
 * (n, n_x, n_y, n_xx, n_xy, n_yy). mode 1: analytic linear velocity c = c1 + gx x + gy y,
 * used only to pin the integrator against a closed form. */
typedef struct {
    int mode;
    int nx, ny;
    double dx, x0, y0;
    const double *f;        /* [6][ny][nx] */
    double c1, gx, gy;
    const double *al;       /* absorption coefficient alpha [ny][nx] in Np/m, NULL: lossless */
    const double *nr;       /* slowness integrated along the rays [ny][nx]; NULL: the traced n */
} og_medium;

typedef struct { double n, gx, gy, hxx, hxy, hyy, al, nr; } fval;

/* ------------------------------------------------------------------ a1 */

/* Odd smoothing window (grid points). The paper quotes windows 13, 11, 9, 7 from low
 * to high frequency on a 1 mm grid, 7 at 1 MHz, and scales the width inversely with the
 * grid spacing (Sec. 6.2, Sec. 6.3.2). Reading: 13 below 0.4 MHz, 11 below 0.7 MHz,
 * 9 below 1 MHz, 7 from 1 MHz; then the nearest odd integer to w * (1 mm / dx). */
int og_window(const og_geom *g, double f)
{
    double w1 = f < 0.4e6 ? 13.0 : (f < 0.7e6 ? 11.0 : (f < 1.0e6 ? 9.0 : 7.0));
    double w = w1 * (1e-3 / g->dx);
    int k = (int)floor((w - 1.0) / 2.0 + 0.5);   /* nearest odd 2k+1 */
    if (k < 0) k = 0;
    return 2 * k + 1;
}

static int clampi(int i, int lo, int hi) { return i < lo ? lo : (i > hi ? hi : i); }

/* Separable moving average of width w on the slowness 1/c, edges replicated. */
void og_smooth(const og_geom *g, const double *c, int w, double *ns)
{
    int nx = g->nx, ny = g->ny, h = (w - 1) / 2;
    double *n = malloc(sizeof(double) * nx * ny), *t = malloc(sizeof(double) * nx * ny);
    for (int k = 0; k < nx * ny; k++) n[k] = 1.0 / c[k];
    for (int iy = 0; iy < ny; iy++)
        for (int ix = 0; ix < nx; ix++) {
            double s = 0;
            for (int d = -h; d <= h; d++) s += n[iy * nx + clampi(ix + d, 0, nx - 1)];
            t[iy * nx + ix] = s / w;
        }
    for (int iy = 0; iy < ny; iy++)
        for (int ix = 0; ix < nx; ix++) {
            double s = 0;
            for (int d = -h; d <= h; d++) s += t[clampi(iy + d, 0, ny - 1) * nx + ix];
            ns[iy * nx + ix] = s / w;
        }
    free(n);
    free(t);
}

/* Separable moving average of width w of an arbitrary map, edges replicated (the same
 * filter as og_smooth). */
static void box_smooth(const og_geom *g, const double *in, int w, double *out)
{
    int h = w / 2, nx = g->nx, ny = g->ny;
    double *t = malloc(sizeof(double) * nx * ny);
    for (int iy = 0; iy < ny; iy++)
        for (int ix = 0; ix < nx; ix++) {
            double s = 0;
            for (int d = -h; d <= h; d++) s += in[iy * nx + clampi(ix + d, 0, nx - 1)];
            t[iy * nx + ix] = s / w;
        }
    for (int iy = 0; iy < ny; iy++)
        for (int ix = 0; ix < nx; ix++) {
            double s = 0;
            for (int d = -h; d <= h; d++) s += t[clampi(iy + d, 0, ny - 1) * nx + ix];
            out[iy * nx + ix] = s / w;
        }
    free(t);
}

/* Smoothing with absorption (Sec. 6.2: the wavenumber map is smoothed before tracing).
 * Reading: the complex wavenumber map k~ / omega = n_e + i alpha0 omega^(y-1) is smoothed
 * by the same window, i.e. both the ray slowness n_e = 1/c + alpha0 tan(pi y/2) omega^(y-1)
 * (Eq. wave-number) and the absorption coefficient alpha = alpha0 omega^y. Outputs:
 * ns = smoothed 1/c (the smooth background of the Born split, m_s = ns^2), ne = smoothed
 * n_e (the field the rays follow), as = smoothed alpha (Np/m). alpha0 in Np (rad/s)^-y m^-1. */
void og_smooth_abs(const og_geom *g, const double *c, const double *alpha0, double y, double f, int w, double *ns,
                   double *ne, double *as)
{
    size_t P = (size_t)g->nx * g->ny;
    double om = 2 * M_PI * f, tn = tan(M_PI * y / 2) * pow(om, y - 1), wy = pow(om, y);
    double *a = malloc(sizeof(double) * P), *b = malloc(sizeof(double) * P), *q = malloc(sizeof(double) * P);
    for (size_t k = 0; k < P; k++) {
        a[k] = 1.0 / c[k];
        b[k] = 1.0 / c[k] + alpha0[k] * tn;
        q[k] = alpha0[k] * wy;
    }
    box_smooth(g, a, w, ns);
    box_smooth(g, b, w, ne);
    box_smooth(g, q, w, as);
    free(a); free(b); free(q);
}

/* Central differences of the smoothed slowness (edge indices clamped). */
void og_fields(const og_geom *g, const double *ns, double *f)
{
    int nx = g->nx, ny = g->ny;
    double dx = g->dx;
    size_t P = (size_t)nx * ny;
#define NS(ix, iy) ns[clampi(iy, 0, ny - 1) * nx + clampi(ix, 0, nx - 1)]
    for (int iy = 0; iy < ny; iy++)
        for (int ix = 0; ix < nx; ix++) {
            size_t k = (size_t)iy * nx + ix;
            f[k] = NS(ix, iy);
            f[P + k] = (NS(ix + 1, iy) - NS(ix - 1, iy)) / (2 * dx);
            f[2 * P + k] = (NS(ix, iy + 1) - NS(ix, iy - 1)) / (2 * dx);
            f[3 * P + k] = (NS(ix + 1, iy) - 2 * NS(ix, iy) + NS(ix - 1, iy)) / (dx * dx);
            f[4 * P + k] = (NS(ix + 1, iy + 1) - NS(ix - 1, iy + 1) - NS(ix + 1, iy - 1) + NS(ix - 1, iy - 1)) /
                           (4 * dx * dx);
            f[5 * P + k] = (NS(ix, iy + 1) - 2 * NS(ix, iy) + NS(ix, iy - 1)) / (dx * dx);
        }
#undef NS
}

/* Row-major indices of the nodes inside the reconstruction mask |x| <= mask_r (Sec. 6.3). */
int og_mask(const og_geom *g, int *idx)
{
    int X = 0;
    for (int iy = 0; iy < g->ny; iy++)
        for (int ix = 0; ix < g->nx; ix++) {
            double x = g->x0 + ix * g->dx, y = g->y0 + iy * g->dx;
            if (x * x + y * y <= g->mask_r * g->mask_r) {
                if (idx) idx[X] = iy * g->nx + ix;
                X++;
            }
        }
    return X;
}

/* Grid-to-ray interpolation (Sec. 4.4). Reading: bilinear interpolation of the six
 * precomputed derivative fields (the paper uses B-splines). */
static void field_eval(const og_medium *m, double px, double py, fval *o)
{
    if (m->mode == 1) {
        double c = m->c1 + m->gx * px + m->gy * py;
        o->n = 1.0 / c;
        o->gx = -m->gx / (c * c);
        o->gy = -m->gy / (c * c);
        o->hxx = 2 * m->gx * m->gx / (c * c * c);
        o->hxy = 2 * m->gx * m->gy / (c * c * c);
        o->hyy = 2 * m->gy * m->gy / (c * c * c);
        o->al = 0;
        o->nr = o->n;
        return;
    }
    double u = (px - m->x0) / m->dx, v = (py - m->y0) / m->dx;
    int i = clampi((int)floor(u), 0, m->nx - 2), j = clampi((int)floor(v), 0, m->ny - 2);
    double tx = u - i, ty = v - j;
    double w00 = (1 - tx) * (1 - ty), w10 = tx * (1 - ty), w01 = (1 - tx) * ty, w11 = tx * ty;
    size_t P = (size_t)m->nx * m->ny, k = (size_t)j * m->nx + i;
    double r[6];
    for (int q = 0; q < 6; q++) {
        const double *F = m->f + q * P;
        r[q] = w00 * F[k] + w10 * F[k + 1] + w01 * F[k + m->nx] + w11 * F[k + m->nx + 1];
    }
    o->n = r[0]; o->gx = r[1]; o->gy = r[2]; o->hxx = r[3]; o->hxy = r[4]; o->hyy = r[5];
    o->al = 0;
    if (m->al) {
        const double *F = m->al;
        o->al = w00 * F[k] + w10 * F[k + 1] + w01 * F[k + m->nx] + w11 * F[k + m->nx + 1];
    }
    o->nr = o->n;
    if (m->nr) {
        const double *F = m->nr;
        o->nr = w00 * F[k] + w10 * F[k + 1] + w01 * F[k + m->nx] + w11 * F[k + m->nx + 1];
    }
}

/* ------------------------------------------------------------------ a2 */

/* One ray sample. J is det[dx/d gamma0, dx/ds] from the paraxial dx and the unit
 * direction; a is the reduced amplitude of Eq. amplitude-geom-discretised:
 * A_geom = (8 pi omega / c0)^(-1/2) * a, a_i = [ (c_i / c_1) |J_1 / J_i| / ds ]^(1/2),
 * with the reference amplitude [8 pi k0 |x_1 - x_0|]^(-1/2) and |x_1 - x_0| = ds. */
typedef struct {
    double x, y, T, J, a, gam, n, dH, px, py, B;
    int K;
} osample;

#define SAMPLE_DOUBLES 13

/* Trace one ray from (xs,ys) with initial direction gam0 until it crosses radius R.
 * Samples 0..M are written to out (M returned), -1 if maxs steps are exceeded.
 *
 * Alg. 1 in slowness variables: with k = omega n the ray path and the paraxial
 * system do not depend on omega, so p = k / omega and dp = dk / omega are carried.
 * Reading of Alg. 1: both stages of the paraxial update use the reference-ray
 * quantities of the same stage (p, grad n, Hess n at x; p', grad n', Hess n' at
 * x + ds q_x). Travel time is the trapezoid rule of n along the samples (of the unsmoothed
 * slowness when the medium carries one, Sec. 6.3.2: rays traced on the smoothed map,
 * integration on the non-smoothed one; the amplitude's c ratio likewise); with absorption
 * B = int alpha ds uses the same rule and the sample amplitude is a exp(-B) (A = A_abs A_geom,
 * Eqs. amplitude-abs-discretised, amplitude-geom-discretised). */
int og_trace_ray(const og_medium *m, double R, double ds, double xs, double ys, double gam0, int maxs,
                 osample *out)
{
    fval F, G, H;
    field_eval(m, xs, ys, &F);
    double x = xs, y = ys, n = F.n;
    double px = n * cos(gam0), py = n * sin(gam0);
    /* paraxial initial condition: dx = 0, p . dp = 0 (Sec. 4.4, initial conditions) */
    double dxx = 0, dxy = 0, dpx = -n * sin(gam0), dpy = n * cos(gam0);
    double T = 0, B = 0;
    int K = 0;
    double J1 = 0, n1 = 0, Jlast = 0;
    memset(&out[0], 0, sizeof(osample));
    out[0].x = x; out[0].y = y; out[0].n = n; out[0].gam = gam0; out[0].px = px; out[0].py = py;
    for (int i = 0; i < maxs; i++) {
        /* reference ray, stage 1 (normalise, update variables) */
        field_eval(m, x, y, &F);
        n = F.n;
        double pn = sqrt(px * px + py * py);
        px *= n / pn; py *= n / pn;
        double qx = px / n, qy = py / n, qpx = F.gx, qpy = F.gy;
        /* auxiliary point */
        double xa = x + ds * qx, ya = y + ds * qy;
        field_eval(m, xa, ya, &G);
        double pax = px + ds * qpx, pay = py + ds * qpy;
        double pan = sqrt(pax * pax + pay * pay);
        pax *= G.n / pan; pay *= G.n / pan;
        double qax = pax / G.n, qay = pay / G.n, qpax = G.gx, qpay = G.gy;
        /* position update along the normalised mean direction; wavevector update */
        double sx = qx + qax, sy = qy + qay, sn = sqrt(sx * sx + sy * sy);
        double dirx = sx / sn, diry = sy / sn;
        double xn = x + ds * dirx, yn = y + ds * diry;
        double pxn = px + ds * (qpx + qpax) / 2, pyn = py + ds * (qpy + qpay) / 2;
        /* paraxial ray: q_dx = -n^-2 p (grad n . dx) + dp / n,
         *               q_dp = Hess n dx - grad n (grad n . dx) / n + grad n (p . dp) / n^2 */
        double gd = F.gx * dxx + F.gy * dxy, pd = px * dpx + py * dpy;
        double qdxx = -px * gd / (n * n) + dpx / n, qdxy = -py * gd / (n * n) + dpy / n;
        double qdpx = F.hxx * dxx + F.hxy * dxy - F.gx * gd / n + F.gx * pd / (n * n);
        double qdpy = F.hxy * dxx + F.hyy * dxy - F.gy * gd / n + F.gy * pd / (n * n);
        double dpax = dpx + ds * qdpx, dpay = dpy + ds * qdpy;
        double dxax = dxx + ds * qdxx, dxay = dxy + ds * qdxy;
        double gda = G.gx * dxax + G.gy * dxay, pda = pax * dpax + pay * dpay;
        double qdxax = -pax * gda / (G.n * G.n) + dpax / G.n, qdxay = -pay * gda / (G.n * G.n) + dpay / G.n;
        double qdpax = G.hxx * dxax + G.hxy * dxay - G.gx * gda / G.n + G.gx * pda / (G.n * G.n);
        double qdpay = G.hxy * dxax + G.hyy * dxay - G.gy * gda / G.n + G.gy * pda / (G.n * G.n);
        double dxxn = dxx + ds * (qdxx + qdxax) / 2, dxyn = dxy + ds * (qdxy + qdxay) / 2;
        double dpxn = dpx + ds * (qdpx + qdpax) / 2, dpyn = dpy + ds * (qdpy + qdpay) / 2;
        field_eval(m, xn, yn, &H);
        double Tn = T + ds * (F.nr + H.nr) / 2, Bn = B + ds * (F.al + H.al) / 2;
        int last = 0;
        if (xn * xn + yn * yn >= R * R) {
            /* final partial step ds' <= ds landing on the ring (Def. ray-parameterisation):
             * the crossing of the step's chord with the ring; the other ray quantities are
             * interpolated linearly along the chord. */
            double b = x * dirx + y * diry, cc = x * x + y * y - R * R;
            double disc = b * b - cc;
            double t = -b + sqrt(disc > 0 ? disc : 0);
            if (t > ds) t = ds;
            if (t < 0) t = 0;
            double fr = t / ds;
            xn = x + t * dirx; yn = y + t * diry;
            Tn = T + fr * (Tn - T);
            Bn = B + fr * (Bn - B);
            dxxn = dxx + fr * (dxxn - dxx); dxyn = dxy + fr * (dxyn - dxy);
            dpxn = dpx + fr * (dpxn - dpx); dpyn = dpy + fr * (dpyn - dpy);
            pxn = px + fr * (pxn - px); pyn = py + fr * (pyn - py);
            field_eval(m, xn, yn, &H);
            last = 1;
        }
        x = xn; y = yn; px = pxn; py = pyn; dxx = dxxn; dxy = dxyn; dpx = dpxn; dpy = dpyn; T = Tn; B = Bn;
        /* sample i+1 */
        double pm = sqrt(px * px + py * py), tx = px / pm, ty = py / pm;
        double J = dxx * ty - dxy * tx;
        if (i == 0) { J1 = J; n1 = H.nr; Jlast = J; }
        else if (J * Jlast < 0) { K++; }   /* caustic: sign change of the ray Jacobian */
        if (J != 0) Jlast = J;
        osample *s = &out[i + 1];
        s->x = x; s->y = y; s->T = T; s->J = J; s->n = H.n; s->px = px; s->py = py; s->K = K;
        s->gam = atan2(py, px);
        s->a = sqrt((n1 / H.nr) * fabs(J1 / J) / ds) * exp(-B);
        s->B = B;
        /* paraxial condition dH = grad_p H . dp + grad_x H . dx, H = (p.p - n^2) / (2n) */
        double pp = px * px + py * py;
        double hx = -H.gx * (pp + H.n * H.n) / (2 * H.n * H.n), hy = -H.gy * (pp + H.n * H.n) / (2 * H.n * H.n);
        s->dH = (px * dpx + py * dpy) / H.n + hx * dxx + hy * dxy;
        if (last) return i + 1;
    }
    return -1;
}

/* Flat-array wrapper used by the tests: rows of SAMPLE_DOUBLES doubles
 * (x, y, T, J, a, gamma, K, n, dH, px, py, s, B). */
int og_trace_ray_flat(const og_medium *m, double R, double ds, double xs, double ys, double gam0, int maxs,
                      double *rows)
{
    osample *s = malloc(sizeof(osample) * (maxs + 1));
    int M = og_trace_ray(m, R, ds, xs, ys, gam0, maxs, s);
    int cnt = M < 0 ? maxs + 1 : M + 1;
    for (int i = 0; i < cnt; i++) {
        double *r = rows + (size_t)i * SAMPLE_DOUBLES;
        r[0] = s[i].x; r[1] = s[i].y; r[2] = s[i].T; r[3] = s[i].J; r[4] = s[i].a; r[5] = s[i].gam;
        r[6] = s[i].K; r[7] = s[i].n; r[8] = s[i].dH; r[9] = s[i].px; r[10] = s[i].py; r[12] = s[i].B;
        r[11] = (i == M && M > 0) ? (M - 1) * ds + sqrt((s[i].x - s[i - 1].x) * (s[i].x - s[i - 1].x) +
                                                        (s[i].y - s[i - 1].y) * (s[i].y - s[i - 1].y))
                                  : i * ds;
    }
    free(s);
    return M;
}

/* ------------------------------------------------------------------ a3 */

typedef struct { double x, y, T, a, kx, ky; int K; long id; } vtx;

/* Edge function of the directed edge P->Q at point p, always evaluated from the
 * vertex with the smaller id so that two triangles sharing an edge see exactly
 * opposite values (no node falls between them). */
static double edge_fn(const vtx *P, const vtx *Q, double px, double py)
{
    if (P->id < Q->id) return (Q->x - P->x) * (py - P->y) - (Q->y - P->y) * (px - P->x);
    return -((P->x - Q->x) * (py - Q->y) - (P->y - Q->y) * (px - Q->x));
}

typedef struct {
    double *T, *a, *gam; int *K;   /* per mask node of one fan */
    long *key;                      /* winning triangle (j, i, which) packed; -1 = none */
} fan_out;

/* Rasterise triangle (A,B,C) with key into the fan's tables: barycentric T, a,
 * direction kappa (renormalised through atan2), K = max over the vertices.
 * Overlaps keep the smallest T, ties the smallest key (reading of the paper's
 * triangulation / interpolation of ray quantities onto the grid, Sec. 4.4). */
static void raster_tri(const og_geom *g, const int *node2x, const vtx *A, const vtx *B, const vtx *C, long key,
                       fan_out *o)
{
    double ar = (B->x - A->x) * (C->y - A->y) - (B->y - A->y) * (C->x - A->x);
    if (fabs(ar) <= 1e-9 * g->ds * g->ds) return;   /* degenerate */
    double minx = fmin(A->x, fmin(B->x, C->x)), maxx = fmax(A->x, fmax(B->x, C->x));
    double miny = fmin(A->y, fmin(B->y, C->y)), maxy = fmax(A->y, fmax(B->y, C->y));
    int ix0 = (int)ceil((minx - g->x0) / g->dx), ix1 = (int)floor((maxx - g->x0) / g->dx);
    int iy0 = (int)ceil((miny - g->y0) / g->dx), iy1 = (int)floor((maxy - g->y0) / g->dx);
    if (ix0 < 0) ix0 = 0;
    if (iy0 < 0) iy0 = 0;
    if (ix1 > g->nx - 1) ix1 = g->nx - 1;
    if (iy1 > g->ny - 1) iy1 = g->ny - 1;
    for (int iy = iy0; iy <= iy1; iy++)
        for (int ix = ix0; ix <= ix1; ix++) {
            int xi = node2x[iy * g->nx + ix];
            if (xi < 0) continue;
            double px = g->x0 + ix * g->dx, py = g->y0 + iy * g->dx;
            double eA = edge_fn(B, C, px, py), eB = edge_fn(C, A, px, py), eC = edge_fn(A, B, px, py);
            double sum = eA + eB + eC;
            int in = sum > 0 ? (eA >= 0 && eB >= 0 && eC >= 0) : (eA <= 0 && eB <= 0 && eC <= 0);
            if (!in || sum == 0) continue;
            double la = eA / sum, lb = eB / sum, lc = eC / sum;
            double T = la * A->T + lb * B->T + lc * C->T;
            if (o->key[xi] >= 0 && !(T < o->T[xi] || (T == o->T[xi] && key < o->key[xi]))) continue;
            o->T[xi] = T;
            o->a[xi] = la * A->a + lb * B->a + lc * C->a;
            double kx = la * A->kx + lb * B->kx + lc * C->kx, ky = la * A->ky + lb * B->ky + lc * C->ky;
            o->gam[xi] = atan2(ky, kx);
            int K = A->K > B->K ? A->K : B->K;
            o->K[xi] = K > C->K ? K : C->K;
            o->key[xi] = key;
        }
}

static int max_steps(const og_geom *g) { return (int)ceil(3.0 * g->R / g->ds) + 8; }

/* Ray fan of transducer e (a2): N-1 rays j = 1..N-1 leaving x_e at gamma0 = beta_e + pi/2
 * + pi j / N, i.e. at psi_j = -pi/2 + pi j / N from the inward normal, so that on the
 * uniform ring ray j reaches receiver e + j in water (reading of the paper's ray linking for
 * a full ring; the fan replaces per-pair linking). Other positions on the ring keep the same
 * fan; the direct term then interpolates between the rays that bracket each receiver. Rays stop on the ring (radius R). Then (a3) the quad
 * between rays j, j+1 and samples i, i+1 (i >= 1) is split into triangles
 * (P[j,i], P[j+1,i], P[j+1,i+1]) and (P[j,i], P[j+1,i+1], P[j,i+1]) and rasterised.
 * exits[(j-1)*4 + {0,1,2,3}] = (exit angle, T, a, K) of ray j on the ring.
 * Returns 0, or the number of rays that did not reach the ring. */
static int fan_tables(const og_geom *g, const og_medium *med, const int *node2x, int e, fan_out *o, double *exits)
{
    int N = g->N, maxs = max_steps(g), bad = 0;
    double be = xducer_angle(g, e), xe = g->R * cos(be), ye = g->R * sin(be);
    osample *prev = malloc(sizeof(osample) * (maxs + 1)), *cur = malloc(sizeof(osample) * (maxs + 1));
    int Mprev = -1;
    for (int j = 1; j <= N - 1; j++) {
        double gam0 = be + M_PI / 2 + M_PI * j / N;
        int M = og_trace_ray(med, g->R, g->ds, xe, ye, gam0, maxs, cur);
        if (M < 0) { bad++; M = maxs; }
        osample *L = &cur[M];
        exits[(j - 1) * 4 + 0] = atan2(L->y, L->x);
        exits[(j - 1) * 4 + 1] = L->T;
        exits[(j - 1) * 4 + 2] = L->a;
        exits[(j - 1) * 4 + 3] = L->K;
        if (j >= 2) {
            int Mq = Mprev < M ? Mprev : M;
            for (int i = 1; i <= Mq - 1; i++) {
                vtx P00, P01, P10, P11;
                const osample *s[4] = {&prev[i], &prev[i + 1], &cur[i], &cur[i + 1]};
                vtx *v[4] = {&P00, &P01, &P10, &P11};
                int jj[4] = {j - 1, j - 1, j, j}, ii[4] = {i, i + 1, i, i + 1};
                for (int q = 0; q < 4; q++) {
                    v[q]->x = s[q]->x; v[q]->y = s[q]->y; v[q]->T = s[q]->T; v[q]->a = s[q]->a;
                    v[q]->kx = cos(s[q]->gam); v[q]->ky = sin(s[q]->gam); v[q]->K = s[q]->K;
                    v[q]->id = (long)jj[q] * 1000000L + ii[q];
                }
                long base = ((long)(j - 1) * 1000000L + i) * 2;
                raster_tri(g, node2x, &P00, &P10, &P11, base, o);
                raster_tri(g, node2x, &P00, &P11, &P01, base + 1, o);
            }
        }
        osample *t = prev; prev = cur; cur = t;
        Mprev = M;
    }
    free(prev);
    free(cur);
    return bad;
}

/* Tables of the fans listed in fans[0..nf-1] (all fans when fans == NULL, nf = N).
 * Row q of each output (X entries) belongs to fan fans[q]. Uncovered mask nodes get
 * T = 0, a = 0, gamma = 0, K = 0 and covered = 0. Returns the number of uncovered
 * (fan, node) entries; *bad_rays counts rays that never reached the ring. */
long og_tables_ext(const og_geom *g, const double *f6, const double *al, const double *nr, const int *fans, int nf,
                   double *T, double *a, double *gam, int *K, int *covered, double *exits, long *bad_rays);

long og_tables_abs(const og_geom *g, const double *f6, const double *al, const int *fans, int nf, double *T,
                   double *a, double *gam, int *K, int *covered, double *exits, long *bad_rays)
{
    return og_tables_ext(g, f6, al, NULL, fans, nf, T, a, gam, K, covered, exits, bad_rays);
}

long og_tables(const og_geom *g, const double *f6, const int *fans, int nf, double *T, double *a, double *gam,
               int *K, int *covered, double *exits, long *bad_rays)
{
    return og_tables_abs(g, f6, NULL, fans, nf, T, a, gam, K, covered, exits, bad_rays);
}

/* og_tables on a lossy medium: al = absorption coefficient alpha [ny][nx] (Np/m), NULL for a
 * lossless one (the tables' a then holds A_geom A_abs / (8 pi omega / c0)^(-1/2)); nr = slowness
 * integrated along the rays (NULL: the traced, smoothed one). */
long og_tables_ext(const og_geom *g, const double *f6, const double *al, const double *nr, const int *fans, int nf,
                   double *T, double *a, double *gam, int *K, int *covered, double *exits, long *bad_rays)
{
    int X = og_mask(g, NULL);
    int *idx = malloc(sizeof(int) * X), *node2x = malloc(sizeof(int) * g->nx * g->ny);
    og_mask(g, idx);
    for (int k = 0; k < g->nx * g->ny; k++) node2x[k] = -1;
    for (int k = 0; k < X; k++) node2x[idx[k]] = k;
    og_medium med = {0, g->nx, g->ny, g->dx, g->x0, g->y0, f6, 0, 0, 0, al, nr};
    long unc = 0, bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : unc, bad)
    for (int q = 0; q < nf; q++) {
        int e = fans ? fans[q] : q;
        fan_out o;
        size_t off = (size_t)q * X;
        o.T = T + off; o.a = a + off; o.gam = gam + off; o.K = K + off;
        o.key = malloc(sizeof(long) * X);
        for (int k = 0; k < X; k++) { o.key[k] = -1; o.T[k] = 0; o.a[k] = 0; o.gam[k] = 0; o.K[k] = 0; }
        bad += fan_tables(g, &med, node2x, e, &o, exits + (size_t)q * (g->N - 1) * 4);
        for (int k = 0; k < X; k++) {
            covered[off + k] = o.key[k] >= 0;
            if (o.key[k] < 0) unc++;
        }
        free(o.key);
    }
    free(idx);
    free(node2x);
    if (bad_rays) *bad_rays = bad;
    return unc;
}

/* ------------------------------------------------------------------ a4 */

/* |d gamma(x,e) / d e| Delta e by a central difference over the neighbouring
 * transducers, wrapped to (-pi, pi]: dg_e = |wrap(gamma_{e+1} - gamma_{e-1})| / 2.
 * Needs the tables of all N fans; zero where either neighbour is uncovered. */
void og_dgamma(const og_geom *g, int X, const double *gam, const int *covered, double *dg)
{
    int N = g->N;
#pragma omp parallel for
    for (int e = 0; e < N; e++) {
        int ep = (e + 1) % N, em = (e + N - 1) % N;
        for (int k = 0; k < X; k++) {
            size_t ip = (size_t)ep * X + k, im = (size_t)em * X + k;
            if (!covered[ip] || !covered[im]) { dg[(size_t)e * X + k] = 0; continue; }
            double d = gam[ip] - gam[im];
            d = d - 2 * M_PI * floor((d + M_PI) / (2 * M_PI));
            dg[(size_t)e * X + k] = fabs(d) / 2;
        }
    }
}

/* ------------------------------------------------------------------ a5 */

static double wrap2pi(double t) { return t - 2 * M_PI * floor(t / (2 * M_PI)); }

/* Direct Green's function g(omega, r, e) at the receivers, emitter-major g[e*N + r]
 * (complex, interleaved). Reading of ray linking (Sec. 4.4, Sec. 6.3.2): the ray
 * quantities at the ring are interpolated linearly in exit angle between the first
 * pair of consecutive rays j, j+1 (in j order) whose exit angles bracket beta_r;
 * when no pair brackets it, the ray whose exit angle is nearest is used (ties: lower j).
 * K is taken from the nearer ray. g = (8 pi omega/c0)^(-1/2) a exp(i[omega T - pi K/2 + pi/4])
 * (Eqs. 2D_greens, attenuation_geom_reference, phase-discretised). The diagonal is 0.
 * Returns the number of clamped (e, r) pairs. */
long og_direct_green(const og_geom *g, double f, const double *exits_all, double *out)
{
    int N = g->N;
    double w = 2 * M_PI * f, C = 1.0 / sqrt(8 * M_PI * w / g->c0);
    long clamped = 0;
#pragma omp parallel for reduction(+ : clamped)
    for (int e = 0; e < N; e++) {
        const double *ex = exits_all + (size_t)e * (N - 1) * 4;
        double be = xducer_angle(g, e);
        for (int r = 0; r < N; r++) {
            double *o = out + 2 * ((size_t)e * N + r);
            if (r == e) { o[0] = o[1] = 0; continue; }
            double t = wrap2pi(xducer_angle(g, r) - be);
            int found = -1;
            double fr = 0;
            for (int j = 1; j <= N - 2; j++) {
                double tj = wrap2pi(ex[(j - 1) * 4] - be), tk = wrap2pi(ex[j * 4] - be);
                if (tj == tk) continue;
                if ((tj <= t && t <= tk) || (tk <= t && t <= tj)) { found = j; fr = (t - tj) / (tk - tj); break; }
            }
            double T, a;
            int K;
            if (found > 0) {
                const double *A = ex + (found - 1) * 4, *B = ex + found * 4;
                T = A[1] + fr * (B[1] - A[1]);
                a = A[2] + fr * (B[2] - A[2]);
                K = (int)(fr < 0.5 ? A[3] : B[3]);
            } else {
                int best = 1;
                double bd = 1e300;
                for (int j = 1; j <= N - 1; j++) {
                    double d = fabs(wrap2pi(ex[(j - 1) * 4] - be) - t);
                    if (d < bd) { bd = d; best = j; }
                }
                const double *A = ex + (best - 1) * 4;
                T = A[1]; a = A[2]; K = (int)A[3];
                clamped++;
            }
            double ph = w * T - M_PI * K / 2 + M_PI / 4;
            o[0] = C * a * cos(ph);
            o[1] = C * a * sin(ph);
        }
    }
    return clamped;
}

/* Ray linking (Sec. 4.4; Sec. 6.3.2: the secant method on the initial direction of each
 * emitter-receiver pair until the ray meets the receiver within a tolerance). The two fan
 * rays whose exits bracket beta_r (the pair og_direct_green interpolates between) start the
 * secant iteration on the exit angle, kept inside the bracket (regula falsi with the Illinois
 * weighting, so no ray leaves the fan's inward directions); it stops when the exit lies within
 * tol_rad of beta_r (or after maxit rays), and T, a are then interpolated linearly in exit
 * angle between the two bracketing rays to beta_r exactly (K from the nearer). Without a
 * bracket the nearest fan ray is used, as in og_direct_green. Returns the number of such clamped pairs; *unconverged
 * counts pairs that stopped on maxit; T_out (nullable) receives the linked travel times. */
long og_direct_green_linked(const og_geom *g, const og_medium *med, double f, const double *exits_all, int maxit,
                            double tol_rad, double *out, long *unconverged, double *T_out)
{
    int N = g->N, maxs = (int)ceil(3.0 * g->R / g->ds) + 8;
    double w = 2 * M_PI * f, C = 1.0 / sqrt(8 * M_PI * w / g->c0);
    long clamped = 0, unconv = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : clamped, unconv)
    for (int e = 0; e < N; e++) {
        const double *ex = exits_all + (size_t)e * (N - 1) * 4;
        double be = xducer_angle(g, e), xe = g->R * cos(be), ye = g->R * sin(be);
        osample *buf = malloc(sizeof(osample) * (maxs + 1));
        for (int r = 0; r < N; r++) {
            double *o = out + 2 * ((size_t)e * N + r);
            if (r == e) { o[0] = o[1] = 0; continue; }
            double t = wrap2pi(xducer_angle(g, r) - be);
            int found = -1;
            for (int j = 1; j <= N - 2; j++) {
                double tj = wrap2pi(ex[(j - 1) * 4] - be), tk = wrap2pi(ex[j * 4] - be);
                if (tj == tk) continue;
                if ((tj <= t && t <= tk) || (tk <= t && t <= tj)) { found = j; break; }
            }
            double T, a;
            int K;
            if (found < 0) {
                int best = 1;
                double bd = 1e300;
                for (int j = 1; j <= N - 1; j++) {
                    double d = fabs(wrap2pi(ex[(j - 1) * 4] - be) - t);
                    if (d < bd) { bd = d; best = j; }
                }
                const double *A = ex + (best - 1) * 4;
                T = A[1]; a = A[2]; K = (int)A[3];
                clamped++;
            } else {
                /* bracketing secant (regula falsi, Illinois): a and b always bracket the
                 * receiver's exit angle, so every new ray starts strictly between the two fan
                 * rays (inward) and the exit angle converges superlinearly. f = exit angle - t;
                 * wa, wb are the Illinois-weighted values used only for the next angle. */
                double ga = be + M_PI / 2 + M_PI * found / N, gb = be + M_PI / 2 + M_PI * (found + 1) / N;
                double fa = wrap2pi(ex[(found - 1) * 4] - be) - t, fb = wrap2pi(ex[found * 4] - be) - t;
                double Ta = ex[(found - 1) * 4 + 1], Tb = ex[found * 4 + 1];
                double aa = ex[(found - 1) * 4 + 2], ab = ex[found * 4 + 2];
                int Ka = (int)ex[(found - 1) * 4 + 3], Kb = (int)ex[found * 4 + 3];
                double wa = fa, wb = fb;
                int it = 0, side = 0;
                while (fabs(fa) > tol_rad && fabs(fb) > tol_rad && it < maxit && wb != wa) {
                    double gc = (ga * wb - gb * wa) / (wb - wa);
                    int M = og_trace_ray(med, g->R, g->ds, xe, ye, gc, maxs, buf);
                    if (M < 0) break;
                    const osample *L = &buf[M];
                    double fc = wrap2pi(atan2(L->y, L->x) - be) - t;
                    if (fc > M_PI) fc -= 2 * M_PI;
                    if (fc < -M_PI) fc += 2 * M_PI;
                    it++;
                    if ((fc > 0) == (fb > 0)) {          /* c replaces b */
                        gb = gc; fb = fc; wb = fc; Tb = L->T; ab = L->a; Kb = L->K;
                        if (side == -1) wa /= 2;
                        side = -1;
                    } else {                              /* c replaces a */
                        ga = gc; fa = fc; wa = fc; Ta = L->T; aa = L->a; Ka = L->K;
                        if (side == 1) wb /= 2;
                        side = 1;
                    }
                }
                if (fabs(fa) > tol_rad && fabs(fb) > tol_rad) unconv++;
                double fr = (fb == fa) ? 0.0 : (0.0 - fa) / (fb - fa);   /* exit angle interpolated to t */
                T = Ta + fr * (Tb - Ta);
                a = aa + fr * (ab - aa);
                K = fabs(fa) <= fabs(fb) ? Ka : Kb;
            }
            double ph = w * T - M_PI * K / 2 + M_PI / 4;
            o[0] = C * a * cos(ph);
            o[1] = C * a * sin(ph);
            if (T_out) T_out[(size_t)e * N + r] = T;
        }
        free(buf);
    }
    if (unconverged) *unconverged = unconv;
    return clamped;
}

/* ------------------------------------------------------------------ a6 */

/* G_e[x] = (8 pi omega/c0)^(-1/2) a exp(i[omega T - pi K/2 + pi/4])   (Eq. 2D_greens)
 * gdag_e[x] = 1/G_e[x] = a^-1 (8 pi omega/c0)^(1/2) exp(-i[...])       (Eq. greens-time-reversed)
 * Entries with a = 0 (uncovered) give 0 for both. */
static void green(double w, double c0, double T, double a, int K, double *G, double *Gd)
{
    double C = 1.0 / sqrt(8 * M_PI * w / c0), ph = w * T - M_PI * K / 2 + M_PI / 4;
    if (a == 0) { G[0] = G[1] = Gd[0] = Gd[1] = 0; return; }
    G[0] = C * a * cos(ph); G[1] = C * a * sin(ph);
    Gd[0] = cos(ph) / (C * a); Gd[1] = -sin(ph) / (C * a);
}

/* ------------------------------------------------------------------ a7 */

/* Ray-Born forward D[e*N + r] = sum_x G_r[x] G_e[x] v[x] (Eqs. perturb1, derivative),
 * with v[x] = Upsilon_m dm[x] Delta A supplied by the caller (Upsilon_m = omega^2 for a
 * lossless medium, Eq. scattering-potential). Tables are [N][X]. */
void og_forward(const og_geom *g, double f, int X, const double *T, const double *a, const int *K, const double *v,
                double *D)
{
    int N = g->N;
    double w = 2 * M_PI * f;
    double *G = malloc(sizeof(double) * 2 * (size_t)N * X);
#pragma omp parallel for
    for (int e = 0; e < N; e++)
        for (int k = 0; k < X; k++) {
            size_t i = (size_t)e * X + k;
            double Gd[2];
            green(w, g->c0, T[i], a[i], K[i], &G[2 * i], Gd);
        }
#pragma omp parallel for schedule(dynamic, 1)
    for (int e = 0; e < N; e++)
        for (int r = 0; r < N; r++) {
            double sr = 0, si = 0;
            const double *Ge = G + 2 * (size_t)e * X, *Gr = G + 2 * (size_t)r * X;
            for (int k = 0; k < X; k++) {
                double pr = Gr[2 * k] * Ge[2 * k] - Gr[2 * k + 1] * Ge[2 * k + 1];
                double pi = Gr[2 * k] * Ge[2 * k + 1] + Gr[2 * k + 1] * Ge[2 * k];
                sr += pr * v[k];
                si += pi * v[k];
            }
            D[2 * ((size_t)e * N + r)] = sr;
            D[2 * ((size_t)e * N + r) + 1] = si;
        }
    free(G);
}

/* og_forward with a complex v[x] = Upsilon_m dm[x] Delta A (interleaved re, im), the lossy
 * scattering potential Upsilon_m = omega c k~ (Eq. scattering-potential). */
void og_forward_c(const og_geom *g, double f, int X, const double *T, const double *a, const int *K, const double *v,
                  double *D)
{
    int N = g->N;
    double w = 2 * M_PI * f;
    double *G = malloc(sizeof(double) * 2 * (size_t)N * X);
#pragma omp parallel for
    for (int e = 0; e < N; e++)
        for (int k = 0; k < X; k++) {
            size_t i = (size_t)e * X + k;
            double Gd[2];
            green(w, g->c0, T[i], a[i], K[i], &G[2 * i], Gd);
        }
#pragma omp parallel for schedule(dynamic, 1)
    for (int e = 0; e < N; e++)
        for (int r = 0; r < N; r++) {
            double sr = 0, si = 0;
            const double *Ge = G + 2 * (size_t)e * X, *Gr = G + 2 * (size_t)r * X;
            for (int k = 0; k < X; k++) {
                double pr = Gr[2 * k] * Ge[2 * k] - Gr[2 * k + 1] * Ge[2 * k + 1];
                double pi = Gr[2 * k] * Ge[2 * k + 1] + Gr[2 * k + 1] * Ge[2 * k];
                sr += pr * v[2 * k] - pi * v[2 * k + 1];
                si += pr * v[2 * k + 1] + pi * v[2 * k];
            }
            D[2 * ((size_t)e * N + r)] = sr;
            D[2 * ((size_t)e * N + r) + 1] = si;
        }
    free(G);
}

/* Plain adjoint of og_forward_c: out[x] = dA conj(Upsilon_m[x]) sum_{e,r} conj(G_r G_e) R,
 * ups[x] = Upsilon_m at the listed nodes (interleaved). */
void og_adjoint_plain_c(const og_geom *g, double f, int X, const double *T, const double *a, const int *K,
                        const double *ups, const double *Rm, const int *nodes, int nn, double *out)
{
    int N = g->N;
    double w = 2 * M_PI * f, dA = g->dx * g->dx;
#pragma omp parallel for schedule(dynamic, 16)
    for (int q = 0; q < nn; q++) {
        int k = nodes[q];
        double *G = malloc(sizeof(double) * 2 * N), Gd[2];
        for (int e = 0; e < N; e++) {
            size_t i = (size_t)e * X + k;
            green(w, g->c0, T[i], a[i], K[i], &G[2 * e], Gd);
        }
        double sr = 0, si = 0;
        for (int e = 0; e < N; e++)
            for (int r = 0; r < N; r++) {
                double pr = G[2 * r] * G[2 * e] - G[2 * r + 1] * G[2 * e + 1];
                double pi = G[2 * r] * G[2 * e + 1] + G[2 * r + 1] * G[2 * e];
                const double *R = Rm + 2 * ((size_t)e * N + r);
                sr += pr * R[0] + pi * R[1];
                si += pr * R[1] - pi * R[0];
            }
        double ur = ups[2 * q], ui = -ups[2 * q + 1];
        out[2 * q] = dA * (ur * sr - ui * si);
        out[2 * q + 1] = dA * (ur * si + ui * sr);
        free(G);
    }
}

/* Plain adjoint of og_forward: out[x] = omega^2 dA sum_{e,r} conj(G_r[x] G_e[x]) R[e*N + r]
 * (the Q = 1 gradient of Eq. functional-gradient). nodes: mask indices to evaluate. */
void og_adjoint_plain(const og_geom *g, double f, int X, const double *T, const double *a, const int *K,
                      const double *Rm, const int *nodes, int nn, double *out)
{
    int N = g->N;
    double w = 2 * M_PI * f, dA = g->dx * g->dx;
#pragma omp parallel for schedule(dynamic, 16)
    for (int q = 0; q < nn; q++) {
        int k = nodes[q];
        double *G = malloc(sizeof(double) * 2 * N), Gd[2];
        for (int e = 0; e < N; e++) {
            size_t i = (size_t)e * X + k;
            green(w, g->c0, T[i], a[i], K[i], &G[2 * e], Gd);
        }
        double sr = 0, si = 0;
        for (int e = 0; e < N; e++)
            for (int r = 0; r < N; r++) {
                double pr = G[2 * r] * G[2 * e] - G[2 * r + 1] * G[2 * e + 1];
                double pi = G[2 * r] * G[2 * e + 1] + G[2 * r + 1] * G[2 * e];
                const double *R = Rm + 2 * ((size_t)e * N + r);
                sr += pr * R[0] + pi * R[1];    /* conj(p) * R */
                si += pr * R[1] - pi * R[0];
            }
        out[2 * q] = w * w * dA * sr;
        out[2 * q + 1] = w * w * dA * si;
        free(G);
    }
}

/* ------------------------------------------------------------------ a8 */

/* Preconditioned back-projection, unfactorised (Eqs. sound_speed_update2, btk-amp-angle):
 * out[x] = sum_{e,r} W_er(x) u_e(x) u_r(x) R[e*N + r],  u_e = dg_e gdag_e,
 * where |kbar| |d|kbar|/d omega| / Upsilon_m = 4 cos^2(theta/2) m / omega = 2 (1 + cos theta) m / omega
 * for a lossless medium; the factor m/omega and Delta omega/(2 pi)^3 are applied in og_update.
 * W_er = 2 (1 - cos(gamma_e - gamma_r)) for the scattering angle theta = gamma_r + pi - gamma_e
 * as printed (weight_mode 0), or 2 (1 + cos(gamma_e - gamma_r)) (weight_mode 1, the isochron
 * gradient k_e + k_r, which reproduces the Bessel kernel of App. D).
 * nodes: mask indices to evaluate; out: complex per listed node. */
void og_backproject(const og_geom *g, double f, int X, const double *T, const double *a, const double *gam,
                    const int *K, const double *dg, const double *Rm, const int *nodes, int nn, double *out)
{
    int N = g->N;
    double w = 2 * M_PI * f, sgn = g->weight_mode == 0 ? -1.0 : 1.0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int q = 0; q < nn; q++) {
        int k = nodes[q];
        double *u = malloc(sizeof(double) * 2 * N), *gm = malloc(sizeof(double) * N), G[2], Gd[2];
        for (int e = 0; e < N; e++) {
            size_t i = (size_t)e * X + k;
            green(w, g->c0, T[i], a[i], K[i], G, Gd);
            u[2 * e] = dg[i] * Gd[0];
            u[2 * e + 1] = dg[i] * Gd[1];
            gm[e] = gam[i];
        }
        double sr = 0, si = 0;
        for (int e = 0; e < N; e++)
            for (int r = 0; r < N; r++) {
                double W = 2 * (1 + sgn * cos(gm[e] - gm[r]));
                double pr = u[2 * e] * u[2 * r] - u[2 * e + 1] * u[2 * r + 1];
                double pi = u[2 * e] * u[2 * r + 1] + u[2 * e + 1] * u[2 * r];
                const double *R = Rm + 2 * ((size_t)e * N + r);
                sr += W * (pr * R[0] - pi * R[1]);
                si += W * (pr * R[1] + pi * R[0]);
            }
        out[2 * q] = sr;
        out[2 * q + 1] = si;
        free(u);
        free(gm);
    }
}

/* ------------------------------------------------------------------ a9 */

/* Search direction and update (Eq. sound_speed_update, Sec. 3.4):
 * dm[x] = -(Delta omega / (2 pi)^3) (m[x] / omega) Re grad[x];  m <- m + tau dm on the mask,
 * c = m^(-1/2); outside the mask c = c0 (Sec. 6.3).
 * Reading: the paper's stationarity condition grad F + H dm = 0 with H ~ 2 pi delta fixes
 * the minus sign (the printed search direction omits it). m is the current unsmoothed map.
 * stats: [0] rms dc over the mask, [1] max |dc|, [2] ||dm||_2 over the mask.
 * Returns 0, or 1 if an updated m is not positive. */
int og_update(const og_geom *g, double f, double df, int X, const int *idx, const double *grad_re,
              const double *c_in, double *c_out, double *stats)
{
    double w = 2 * M_PI * f, dw = 2 * M_PI * df, pref = dw / pow(2 * M_PI, 3);
    int bad = 0;
    double s2 = 0, mx = 0, dm2 = 0;
    for (int k = 0; k < g->nx * g->ny; k++) c_out[k] = g->c0;
    for (int q = 0; q < X; q++) {
        int k = idx[q];
        double m = 1.0 / (c_in[k] * c_in[k]);
        double dm = -pref * (m / w) * grad_re[q];
        double mn = m + g->tau * dm;
        if (!(mn > 0)) { bad = 1; mn = m; }
        c_out[k] = 1.0 / sqrt(mn);
        double dc = c_out[k] - c_in[k];
        s2 += dc * dc;
        if (fabs(dc) > mx) mx = fabs(dc);
        dm2 += dm * dm;
    }
    stats[0] = sqrt(s2 / X);
    stats[1] = mx;
    stats[2] = sqrt(dm2);
    return bad;
}

/* Scattering potential Upsilon_m = omega c k~ at a node (Eq. scattering-potential) with
 * k~ = omega/c + alpha0 omega^y (tan(pi y/2) + i) (Eq. szabo_dispersion_equation). */
static void upsilon(double w, double c, double alpha0, double y, double *u)
{
    double al = alpha0 * pow(w, y);
    u[0] = w * c * (w / c + al * tan(M_PI * y / 2));
    u[1] = w * c * al;
}

/* og_update with absorption: the node factor m/omega of the lossless update becomes
 * |kbar| |d|kbar|/d omega| / (4 cos^2(theta/2) Upsilon_m) = k (1/c + y tan(pi y/2) omega^(y-1) alpha0) / Upsilon_m
 * (Eqs. btk-amp-angle and the derivative of |kbar| in Sec. 3.3, Eq. scattering-potential), complex,
 * so dm = -(Delta omega / (2 pi)^3) Re{ factor * grad } with grad the complex unfactorised sum of
 * og_backproject. c and alpha0 are the node's current (unsmoothed) values. */
int og_update_abs(const og_geom *g, double f, double df, int X, const int *idx, const double *grad,
                  const double *c_in, const double *alpha0, double y, double *c_out, double *stats)
{
    double w = 2 * M_PI * f, dw = 2 * M_PI * df, pref = dw / pow(2 * M_PI, 3);
    double tn = tan(M_PI * y / 2);
    int bad = 0;
    double s2 = 0, mx = 0, dm2 = 0;
    for (int k = 0; k < g->nx * g->ny; k++) c_out[k] = g->c0;
    for (int q = 0; q < X; q++) {
        int k = idx[q];
        double c = c_in[k], m = 1.0 / (c * c), a0 = alpha0[k];
        double kr = w / c + a0 * tn * pow(w, y);
        double num = kr * (1.0 / c + y * tn * pow(w, y - 1) * a0);
        double u[2];
        upsilon(w, c, a0, y, u);
        double un = u[0] * u[0] + u[1] * u[1];
        double fr = num * u[0] / un, fi = -num * u[1] / un;           /* num / Upsilon_m */
        double dm = -pref * (fr * grad[2 * q] - fi * grad[2 * q + 1]);
        double mn = m + g->tau * dm;
        if (!(mn > 0)) { bad = 1; mn = m; }
        c_out[k] = 1.0 / sqrt(mn);
        double dc = c_out[k] - c_in[k];
        s2 += dc * dc;
        if (fabs(dc) > mx) mx = fabs(dc);
        dm2 += dm * dm;
    }
    stats[0] = sqrt(s2 / X);
    stats[1] = mx;
    stats[2] = sqrt(dm2);
    return bad;
}

/* ------------------------------------------------------------------ composites */

typedef struct {
    int X;
    int *idx;
    double *f6, *ns, *T, *a, *gam, *dg, *exits;
    double *al, *nr;          /* the medium's alpha and integrated slowness maps (may be NULL) */
    int *K, *cov;
    long uncovered, bad_rays;
} og_state;

static void state_build_abs(const og_geom *g, double f, const double *c, const double *alpha0, double y,
                            og_state *s)
{
    size_t P = (size_t)g->nx * g->ny;
    s->X = og_mask(g, NULL);
    s->idx = malloc(sizeof(int) * s->X);
    og_mask(g, s->idx);
    s->ns = malloc(sizeof(double) * P);
    s->f6 = malloc(sizeof(double) * 6 * P);
    double *ne = NULL, *as = NULL;
    if (alpha0) {
        ne = malloc(sizeof(double) * P);
        as = malloc(sizeof(double) * P);
        og_smooth_abs(g, c, alpha0, y, f, og_window(g, f), s->ns, ne, as);
        og_fields(g, ne, s->f6);
        free(ne);
    } else {
        og_smooth(g, c, og_window(g, f), s->ns);
        og_fields(g, s->ns, s->f6);
    }
    size_t NX = (size_t)g->N * s->X;
    s->T = malloc(sizeof(double) * NX); s->a = malloc(sizeof(double) * NX);
    s->gam = malloc(sizeof(double) * NX); s->dg = malloc(sizeof(double) * NX);
    s->K = malloc(sizeof(int) * NX); s->cov = malloc(sizeof(int) * NX);
    s->exits = malloc(sizeof(double) * (size_t)g->N * (g->N - 1) * 4);
    s->uncovered = og_tables_abs(g, s->f6, as, NULL, g->N, s->T, s->a, s->gam, s->K, s->cov, s->exits,
                                 &s->bad_rays);
    og_dgamma(g, s->X, s->gam, s->cov, s->dg);
    s->al = as;
    s->nr = NULL;
}

static void state_build(const og_geom *g, double f, const double *c, og_state *s)
{
    state_build_abs(g, f, c, NULL, 0.0, s);
}

/* State for the paper's integration (Sec. 6.3.2): rays traced on the smoothed map (as in
 * state_build_abs), travel time, amplitude c ratio and absorption integrated on the
 * non-smoothed maps 1/c and alpha0 omega^y. */
static void state_build_raw(const og_geom *g, double f, const double *c, const double *alpha0, double y, og_state *s)
{
    size_t P = (size_t)g->nx * g->ny;
    s->X = og_mask(g, NULL);
    s->idx = malloc(sizeof(int) * s->X);
    og_mask(g, s->idx);
    s->ns = malloc(sizeof(double) * P);
    s->f6 = malloc(sizeof(double) * 6 * P);
    double *nr = malloc(sizeof(double) * P), *ar = NULL;
    for (size_t k = 0; k < P; k++) nr[k] = 1.0 / c[k];
    if (alpha0) {
        double *ne = malloc(sizeof(double) * P), *as = malloc(sizeof(double) * P);
        og_smooth_abs(g, c, alpha0, y, f, og_window(g, f), s->ns, ne, as);
        og_fields(g, ne, s->f6);
        free(ne);
        free(as);
        ar = malloc(sizeof(double) * P);
        double wy = pow(2 * M_PI * f, y), tn = tan(M_PI * y / 2) * pow(2 * M_PI * f, y - 1);
        for (size_t k = 0; k < P; k++) {
            ar[k] = alpha0[k] * wy;
            nr[k] += alpha0[k] * tn;        /* the real wavenumber over omega, not smoothed */
        }
    } else {
        og_smooth(g, c, og_window(g, f), s->ns);
        og_fields(g, s->ns, s->f6);
    }
    size_t NX = (size_t)g->N * s->X;
    s->T = malloc(sizeof(double) * NX); s->a = malloc(sizeof(double) * NX);
    s->gam = malloc(sizeof(double) * NX); s->dg = malloc(sizeof(double) * NX);
    s->K = malloc(sizeof(int) * NX); s->cov = malloc(sizeof(int) * NX);
    s->exits = malloc(sizeof(double) * (size_t)g->N * (g->N - 1) * 4);
    s->uncovered = og_tables_ext(g, s->f6, ar, nr, NULL, g->N, s->T, s->a, s->gam, s->K, s->cov, s->exits,
                                 &s->bad_rays);
    og_dgamma(g, s->X, s->gam, s->cov, s->dg);
    s->al = ar;
    s->nr = nr;
}

static void state_free(og_state *s)
{
    free(s->idx); free(s->ns); free(s->f6); free(s->T); free(s->a); free(s->gam); free(s->dg);
    free(s->K); free(s->cov); free(s->exits); free(s->al); free(s->nr);
}

#define OG_RAW 1    /* integration on the non-smoothed map, no Born term */
#define OG_LINK 2   /* direct Green's function on secant-linked rays */
#define OG_LINK_MAXIT 8
#define OG_LINK_TOL 1e-6

/* Direct Green's function of a built state: fan interpolation, or linked rays (OG_LINK). */
static long state_direct_green(const og_geom *g, const og_state *s, double f, int opts, double *out)
{
    if (!(opts & OG_LINK)) return og_direct_green(g, f, s->exits, out);
    og_medium med = {0, g->nx, g->ny, g->dx, g->x0, g->y0, s->f6, 0, 0, 0, s->al, s->nr};
    long unc = 0;
    return og_direct_green_linked(g, &med, f, s->exits, OG_LINK_MAXIT, OG_LINK_TOL, out, &unc, NULL) + unc;
}

/* Predicted data g = g_dir + F[m - m_s] on the current model (a5 + a7): the rays are
 * traced on the smoothed map and the rough part m - m_s, m_s = n_s^2, is carried by the
 * Born term. Reading: this is also the data model of the synthetic workloads. stats: [0] uncovered entries, [1] rays not reaching the ring, [2] clamped pairs. */
void og_predict(const og_geom *g, double f, const double *c, double *out, double *stats)
{
    og_state s;
    state_build(g, f, c, &s);
    int N = g->N;
    double w = 2 * M_PI * f, dA = g->dx * g->dx;
    double *v = malloc(sizeof(double) * s.X), *D = malloc(sizeof(double) * 2 * (size_t)N * N);
    for (int q = 0; q < s.X; q++) {
        int k = s.idx[q];
        v[q] = w * w * dA * (1.0 / (c[k] * c[k]) - s.ns[k] * s.ns[k]);
    }
    long cl = og_direct_green(g, f, s.exits, out);
    og_forward(g, f, s.X, s.T, s.a, s.K, v, D);
    for (size_t i = 0; i < 2 * (size_t)N * N; i++) out[i] += D[i];
    for (int e = 0; e < N; e++) out[2 * ((size_t)e * N + e)] = out[2 * ((size_t)e * N + e) + 1] = 0;
    if (stats) { stats[0] = s.uncovered; stats[1] = s.bad_rays; stats[2] = cl; }
    free(v); free(D);
    state_free(&s);
}

/* One Hessian-free update at frequency f with sweep spacing df (a1..a9). data is the
 * measured Green's function [e*N + r]. Residual R = g_pred - data with the diagonal
 * set to 0 (Eq. residual). stats: [0] rms dc, [1] max |dc|, [2] ||dm||, [3] ||R||^2,
 * [4] uncovered entries, [5] rays not reaching the ring, [6] clamped pairs.
 * Returns og_update's status. */
int og_update_frequency(const og_geom *g, double f, double df, const double *c, const double *data, double *c_out,
                        double *stats)
{
    og_state s;
    state_build(g, f, c, &s);
    int N = g->N;
    double w = 2 * M_PI * f, dA = g->dx * g->dx;
    double *v = malloc(sizeof(double) * s.X), *D = malloc(sizeof(double) * 2 * (size_t)N * N);
    double *R = malloc(sizeof(double) * 2 * (size_t)N * N);
    for (int q = 0; q < s.X; q++) {
        int k = s.idx[q];
        v[q] = w * w * dA * (1.0 / (c[k] * c[k]) - s.ns[k] * s.ns[k]);
    }
    long cl = og_direct_green(g, f, s.exits, R);
    og_forward(g, f, s.X, s.T, s.a, s.K, v, D);
    double r2 = 0;
    for (int e = 0; e < N; e++)
        for (int r = 0; r < N; r++) {
            size_t i = 2 * ((size_t)e * N + r);
            if (r == e) { R[i] = R[i + 1] = 0; continue; }
            R[i] += D[i] - data[i];
            R[i + 1] += D[i + 1] - data[i + 1];
            r2 += R[i] * R[i] + R[i + 1] * R[i + 1];
        }
    int *nodes = malloc(sizeof(int) * s.X);
    for (int q = 0; q < s.X; q++) nodes[q] = q;
    double *gr = malloc(sizeof(double) * 2 * s.X), *gre = malloc(sizeof(double) * s.X);
    og_backproject(g, f, s.X, s.T, s.a, s.gam, s.K, s.dg, R, nodes, s.X, gr);
    for (int q = 0; q < s.X; q++) gre[q] = gr[2 * q];
    double st[3];
    int bad = og_update(g, f, df, s.X, s.idx, gre, c, c_out, st);
    stats[0] = st[0]; stats[1] = st[1]; stats[2] = st[2]; stats[3] = r2;
    stats[4] = s.uncovered; stats[5] = s.bad_rays; stats[6] = cl;
    free(v); free(D); free(R); free(nodes); free(gr); free(gre);
    state_free(&s);
    return bad;
}

/* og_predict on a lossy medium (alpha0 [ny][nx], exponent y): rays on the smoothed n_e with
 * the absorbing amplitude, and the Born term with v = Upsilon_m dA (m - m_s), m_s = (smoothed
 * 1/c)^2 (the absorption map is known, not perturbed). */
void og_predict_abs(const og_geom *g, double f, const double *c, const double *alpha0, double y, double *out,
                    double *stats)
{
    og_state s;
    state_build_abs(g, f, c, alpha0, y, &s);
    int N = g->N;
    double w = 2 * M_PI * f, dA = g->dx * g->dx;
    double *v = malloc(sizeof(double) * 2 * s.X), *D = malloc(sizeof(double) * 2 * (size_t)N * N);
    for (int q = 0; q < s.X; q++) {
        int k = s.idx[q];
        double u[2], dm = 1.0 / (c[k] * c[k]) - s.ns[k] * s.ns[k];
        upsilon(w, c[k], alpha0[k], y, u);
        v[2 * q] = u[0] * dA * dm;
        v[2 * q + 1] = u[1] * dA * dm;
    }
    long cl = og_direct_green(g, f, s.exits, out);
    og_forward_c(g, f, s.X, s.T, s.a, s.K, v, D);
    for (size_t i = 0; i < 2 * (size_t)N * N; i++) out[i] += D[i];
    for (int e = 0; e < N; e++) out[2 * ((size_t)e * N + e)] = out[2 * ((size_t)e * N + e) + 1] = 0;
    if (stats) { stats[0] = s.uncovered; stats[1] = s.bad_rays; stats[2] = cl; }
    free(v); free(D);
    state_free(&s);
}

/* og_update_frequency on a lossy medium (see og_predict_abs, og_update_abs). */
int og_update_frequency_abs(const og_geom *g, double f, double df, const double *c, const double *alpha0, double y,
                            const double *data, double *c_out, double *stats)
{
    og_state s;
    state_build_abs(g, f, c, alpha0, y, &s);
    int N = g->N;
    double w = 2 * M_PI * f, dA = g->dx * g->dx;
    double *v = malloc(sizeof(double) * 2 * s.X), *D = malloc(sizeof(double) * 2 * (size_t)N * N);
    double *R = malloc(sizeof(double) * 2 * (size_t)N * N);
    for (int q = 0; q < s.X; q++) {
        int k = s.idx[q];
        double u[2], dm = 1.0 / (c[k] * c[k]) - s.ns[k] * s.ns[k];
        upsilon(w, c[k], alpha0[k], y, u);
        v[2 * q] = u[0] * dA * dm;
        v[2 * q + 1] = u[1] * dA * dm;
    }
    long cl = og_direct_green(g, f, s.exits, R);
    og_forward_c(g, f, s.X, s.T, s.a, s.K, v, D);
    double r2 = 0;
    for (int e = 0; e < N; e++)
        for (int r = 0; r < N; r++) {
            size_t i = 2 * ((size_t)e * N + r);
            if (r == e) { R[i] = R[i + 1] = 0; continue; }
            R[i] += D[i] - data[i];
            R[i + 1] += D[i + 1] - data[i + 1];
            r2 += R[i] * R[i] + R[i + 1] * R[i + 1];
        }
    int *nodes = malloc(sizeof(int) * s.X);
    for (int q = 0; q < s.X; q++) nodes[q] = q;
    double *gr = malloc(sizeof(double) * 2 * s.X);
    og_backproject(g, f, s.X, s.T, s.a, s.gam, s.K, s.dg, R, nodes, s.X, gr);
    double st[3];
    int bad = og_update_abs(g, f, df, s.X, s.idx, gr, c, alpha0, y, c_out, st);
    stats[0] = st[0]; stats[1] = st[1]; stats[2] = st[2]; stats[3] = r2;
    stats[4] = s.uncovered; stats[5] = s.bad_rays; stats[6] = cl;
    free(v); free(D); free(R); free(nodes); free(gr);
    state_free(&s);
    return bad;
}

/* Predicted data. opts = 0 is og_predict / og_predict_abs (g_dir + Born term of the rough part);
 * OG_RAW follows Sec. 6.3.2: g at the ray ends with the phase and amplitude integrated on the
 * non-smoothed map and no Born term (the rough part is already in the phase); OG_LINK takes
 * g_dir on secant-linked rays instead of the fan's exit-angle interpolation. alpha0 may be
 * NULL (lossless). */
void og_predict_ext(const og_geom *g, double f, const double *c, const double *alpha0, double y, int opts,
                    double *out, double *stats)
{
    int raw = opts & OG_RAW;
    if (!raw && !(opts & OG_LINK)) {
        if (alpha0) og_predict_abs(g, f, c, alpha0, y, out, stats);
        else og_predict(g, f, c, out, stats);
        return;
    }
    og_state s;
    if (raw) state_build_raw(g, f, c, alpha0, y, &s);
    else state_build_abs(g, f, c, alpha0, y, &s);
    int N = g->N;
    long cl = state_direct_green(g, &s, f, opts, out);
    if (!raw) {
        double w = 2 * M_PI * f, dA = g->dx * g->dx;
        double *v = malloc(sizeof(double) * 2 * s.X), *D = malloc(sizeof(double) * 2 * (size_t)N * N);
        for (int q = 0; q < s.X; q++) {
            int k = s.idx[q];
            double u[2], d = 1.0 / (c[k] * c[k]) - s.ns[k] * s.ns[k];
            upsilon(w, c[k], alpha0 ? alpha0[k] : 0.0, alpha0 ? y : 1.0, u);
            v[2 * q] = u[0] * dA * d;
            v[2 * q + 1] = u[1] * dA * d;
        }
        og_forward_c(g, f, s.X, s.T, s.a, s.K, v, D);
        for (size_t i = 0; i < 2 * (size_t)N * N; i++) out[i] += D[i];
        free(v);
        free(D);
    }
    for (int e = 0; e < N; e++) out[2 * ((size_t)e * N + e)] = out[2 * ((size_t)e * N + e) + 1] = 0;
    if (stats) { stats[0] = s.uncovered; stats[1] = s.bad_rays; stats[2] = cl; }
    state_free(&s);
}

/* One update from a frequency set (Sec. 6.3.2: two consecutive frequencies per update).
 * Reading: the rays of the set are traced once, on the map smoothed (and, when lossy,
 * dispersed) for the set's first frequency; each frequency f_k of the set contributes its own
 * residual R_k and back-projection, and the search direction is the sum over the set of
 * -(Delta omega/(2 pi)^3) Re{node factor(f_k) grad_k} (Eq. sound_speed_update summed over the
 * set's omega), applied once with the step tau. opts: OG_RAW (the integration of og_predict_ext)
 * and OG_LINK (the direct Green's function on linked rays).
 * data: nf complex [N][N] blocks. stats as og_update_frequency, [3] summed over the set. */
int og_update_set_ext(const og_geom *g, const double *freqs, int nf, double df, const double *c,
                      const double *alpha0, double y, int opts, const double *data, double *c_out, double *stats)
{
    int raw = opts & OG_RAW;
    og_state s;
    if (raw) state_build_raw(g, freqs[0], c, alpha0, y, &s);
    else state_build_abs(g, freqs[0], c, alpha0, y, &s);
    int N = g->N;
    size_t NN = (size_t)N * N;
    double dA = g->dx * g->dx, pref = 2 * M_PI * df / pow(2 * M_PI, 3), tn = tan(M_PI * y / 2);
    double *v = malloc(sizeof(double) * 2 * s.X), *D = malloc(sizeof(double) * 2 * NN);
    double *R = malloc(sizeof(double) * 2 * NN), *gr = malloc(sizeof(double) * 2 * s.X);
    double *dm = calloc(s.X, sizeof(double));
    int *nodes = malloc(sizeof(int) * s.X);
    for (int q = 0; q < s.X; q++) nodes[q] = q;
    double r2 = 0;
    long cl = 0;
    for (int kf = 0; kf < nf; kf++) {
        double f = freqs[kf], w = 2 * M_PI * f;
        cl = state_direct_green(g, &s, f, opts, R);
        if (!raw) {
            for (int q = 0; q < s.X; q++) {
                int k = s.idx[q];
                double u[2], d = 1.0 / (c[k] * c[k]) - s.ns[k] * s.ns[k];
                upsilon(w, c[k], alpha0 ? alpha0[k] : 0.0, alpha0 ? y : 1.0, u);
                v[2 * q] = u[0] * dA * d;
                v[2 * q + 1] = u[1] * dA * d;
            }
            og_forward_c(g, f, s.X, s.T, s.a, s.K, v, D);
        } else {
            memset(D, 0, sizeof(double) * 2 * NN);
        }
        const double *dk = data + 2 * NN * kf;
        for (int e = 0; e < N; e++)
            for (int r = 0; r < N; r++) {
                size_t i = 2 * ((size_t)e * N + r);
                if (r == e) { R[i] = R[i + 1] = 0; continue; }
                R[i] += D[i] - dk[i];
                R[i + 1] += D[i + 1] - dk[i + 1];
                r2 += R[i] * R[i] + R[i + 1] * R[i + 1];
            }
        og_backproject(g, f, s.X, s.T, s.a, s.gam, s.K, s.dg, R, nodes, s.X, gr);
        for (int q = 0; q < s.X; q++) {
            int k = s.idx[q];
            double cc = c[k], m = 1.0 / (cc * cc);
            if (!alpha0) {
                dm[q] += -pref * (m / w) * gr[2 * q];
            } else {
                double a0 = alpha0[k], kr = w / cc + a0 * tn * pow(w, y);
                double num = kr * (1.0 / cc + y * tn * pow(w, y - 1) * a0), u[2];
                upsilon(w, cc, a0, y, u);
                double un = u[0] * u[0] + u[1] * u[1];
                dm[q] += -pref * (num * u[0] / un * gr[2 * q] + num * u[1] / un * gr[2 * q + 1]);
            }
        }
    }
    int bad = 0;
    double s2 = 0, mx = 0, dm2 = 0;
    for (int k = 0; k < g->nx * g->ny; k++) c_out[k] = g->c0;
    for (int q = 0; q < s.X; q++) {
        int k = s.idx[q];
        double m = 1.0 / (c[k] * c[k]), mn = m + g->tau * dm[q];
        if (!(mn > 0)) { bad = 1; mn = m; }
        c_out[k] = 1.0 / sqrt(mn);
        double dc = c_out[k] - c[k];
        s2 += dc * dc;
        if (fabs(dc) > mx) mx = fabs(dc);
        dm2 += dm[q] * dm[q];
    }
    stats[0] = sqrt(s2 / s.X); stats[1] = mx; stats[2] = sqrt(dm2); stats[3] = r2;
    stats[4] = s.uncovered; stats[5] = s.bad_rays; stats[6] = cl;
    free(v); free(D); free(R); free(gr); free(dm); free(nodes);
    state_free(&s);
    return bad;
}

int og_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
