// Steps a2-a5: paraxial ray tracing, ray-to-grid tables, angular density and the
// direct Green's function at the receivers.
//
// Ray fan (reading of the paper's ray linking for a full ring, Sec. 4.4 / 6.3): from
// transducer e, N-1 rays j = 1..N-1 leave at gamma0 = beta_e + pi/2 + pi j / N, so that in
// water ray j reaches receiver e + j. Each ray is integrated by Heun's method with the
// normalisations of Alg. 1 and the paraxial system of Eq. ray-equation-paraxial, in
// slowness variables (p = k / omega, the path does not depend on omega), with step ds and
// a final partial step that lands on the ring (Def. ray-parameterisation).
//
// GB300 mapping: one thread per ray, 32 adjacent rays of one fan per warp stepping in
// lockstep. At each step a lane fetches its neighbour's new sample with a shuffle and
// rasterises the ray-tube quad (rays j, j+1; samples i, i+1) as two triangles straight
// into the fan's table (Sec. 4.4: triangulation of the ray samples). Overlapping triangles
// keep the first arrival: the 16-byte table entry starts with the key (T bits, triangle
// id, K) and a 128-bit compare-and-swap keeps the smallest key, so the table does not
// depend on the order in which warps finish. The ray samples are never stored.
//
// Fields are bilinearly interpolated from the 8-float-per-node field map (L1/L2 cached:
// 8 MB at 512^2). Travel time uses compensated (Kahan) summation.
#include "rbx_internal.cuh"

namespace rbx {

__device__ __forceinline__ int clampi_(int i, int lo, int hi) { return i < lo ? lo : (i > hi ? hi : i); }

struct Fv {
    float n, gx, gy, hxx, hxy, hyy;
};

__device__ __forceinline__ void field_eval(const float *__restrict__ F, const RayParams &p, float px, float py, Fv &o)
{
    float u = (px - p.x0) / p.dx, v = (py - p.y0) / p.dx;
    int i = clampi_((int)floorf(u), 0, p.nx - 2), j = clampi_((int)floorf(v), 0, p.ny - 2);
    float tx = u - (float)i, ty = v - (float)j;
    const float4 *b = reinterpret_cast<const float4 *>(F) + ((size_t)j * p.nx + i) * 2;
    const float4 *c = b + (size_t)p.nx * 2;
    float4 a0 = __ldg(b), a1 = __ldg(b + 1), b0 = __ldg(b + 2), b1 = __ldg(b + 3);
    float4 c0 = __ldg(c), c1 = __ldg(c + 1), d0 = __ldg(c + 2), d1 = __ldg(c + 3);
    float w00 = (1.f - tx) * (1.f - ty), w10 = tx * (1.f - ty), w01 = (1.f - tx) * ty, w11 = tx * ty;
    o.n = w00 * a0.x + w10 * b0.x + w01 * c0.x + w11 * d0.x;
    o.gx = w00 * a0.y + w10 * b0.y + w01 * c0.y + w11 * d0.y;
    o.gy = w00 * a0.z + w10 * b0.z + w01 * c0.z + w11 * d0.z;
    o.hxx = w00 * a0.w + w10 * b0.w + w01 * c0.w + w11 * d0.w;
    o.hxy = w00 * a1.x + w10 * b1.x + w01 * c1.x + w11 * d1.x;
    o.hyy = w00 * a1.y + w10 * b1.y + w01 * c1.y + w11 * d1.y;
}

// A ray sample as a triangle vertex.
struct Vtx {
    float x, y, T, a, kx, ky;
    int K, id;
};

__device__ __forceinline__ void cas128(unsigned long long *addr, unsigned long long clo, unsigned long long chi,
                                       unsigned long long nlo, unsigned long long nhi, unsigned long long &olo,
                                       unsigned long long &ohi)
{
    asm volatile(
        "{\n\t.reg .b128 d, b, c;\n\t"
        "mov.b128 b, {%2, %3};\n\t"
        "mov.b128 c, {%4, %5};\n\t"
        "atom.global.cas.b128 d, [%6], b, c;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(olo), "=l"(ohi)
        : "l"(clo), "l"(chi), "l"(nlo), "l"(nhi), "l"(addr)
        : "memory");
}

__device__ __forceinline__ void load128_cg(const unsigned long long *addr, unsigned long long &lo,
                                           unsigned long long &hi)
{
    asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "l"(addr));
}

// Keep the entry with the smaller key. Each successful exchange lowers the stored key, so
// the loop ends after at most as many rounds as there are competing triangles; the bound
// only guards against a broken invariant and reports it.
__device__ __forceinline__ void cas_min(TabEntry *e, unsigned long long key, unsigned long long pay,
                                        unsigned long long *counters)
{
    unsigned long long *a = reinterpret_cast<unsigned long long *>(e);
    unsigned long long lo, hi;
    load128_cg(a, lo, hi);
    for (int it = 0; it < 1 << 16; ++it) {
        if (key >= lo) return;
        unsigned long long plo, phi;
        cas128(a, lo, hi, key, pay, plo, phi);
        if (plo == lo && phi == hi) return;
        lo = plo;
        hi = phi;
    }
    atomicAdd(&counters[3], 1ull);
}

// Edge function of P->Q at (px,py), evaluated from the vertex with the smaller id so that
// the two triangles sharing an edge see exactly opposite values (watertight).
__device__ __forceinline__ float edge_fn(const Vtx &P, const Vtx &Q, float px, float py)
{
    if (P.id < Q.id) return __fmaf_rn(Q.x - P.x, py - P.y, -__fmul_rn(Q.y - P.y, px - P.x));
    return -__fmaf_rn(P.x - Q.x, py - Q.y, -__fmul_rn(P.y - Q.y, px - Q.x));
}

__device__ void raster_tri(const Vtx &A, const Vtx &B, const Vtx &C, uint32_t tid, const RayParams &p,
                           const int *__restrict__ node2x, TabEntry *fan, unsigned long long *counters)
{
    float ar = (B.x - A.x) * (C.y - A.y) - (B.y - A.y) * (C.x - A.x);
    if (fabsf(ar) <= 1e-9f * p.ds * p.ds) return;  // degenerate
    float minx = fminf(A.x, fminf(B.x, C.x)), maxx = fmaxf(A.x, fmaxf(B.x, C.x));
    float miny = fminf(A.y, fminf(B.y, C.y)), maxy = fmaxf(A.y, fmaxf(B.y, C.y));
    int ix0 = max(0, (int)ceilf((minx - p.x0) / p.dx)), ix1 = min(p.nx - 1, (int)floorf((maxx - p.x0) / p.dx));
    int iy0 = max(0, (int)ceilf((miny - p.y0) / p.dx)), iy1 = min(p.ny - 1, (int)floorf((maxy - p.y0) / p.dx));
    for (int iy = iy0; iy <= iy1; iy++) {
        float py = p.y0 + (float)iy * p.dx;
        for (int ix = ix0; ix <= ix1; ix++) {
            int xi = __ldg(&node2x[iy * p.nx + ix]);
            if (xi < 0) continue;
            float px = p.x0 + (float)ix * p.dx;
            float eA = edge_fn(B, C, px, py), eB = edge_fn(C, A, px, py), eC = edge_fn(A, B, px, py);
            float sum = eA + eB + eC;
            bool in = sum > 0.f ? (eA >= 0.f && eB >= 0.f && eC >= 0.f) : (eA <= 0.f && eB <= 0.f && eC <= 0.f);
            if (!in || sum == 0.f) continue;
            float lb = eB / sum, lc = eC / sum, la = eA / sum;
            float T = A.T + lb * (B.T - A.T) + lc * (C.T - A.T);
            float a = la * A.a + lb * B.a + lc * C.a;
            float kx = la * A.kx + lb * B.kx + lc * C.kx, ky = la * A.ky + lb * B.ky + lc * C.ky;
            float gam = atan2f(ky, kx);
            int K = max(A.K, max(B.K, C.K));
            unsigned long long key = ((unsigned long long)__float_as_uint(T) << 32) | ((unsigned long long)tid << 8) |
                                     (unsigned long long)min(K, 255);
            unsigned long long pay = ((unsigned long long)__float_as_uint(gam) << 32) | __float_as_uint(a);
            cas_min(&fan[xi], key, pay, counters);
        }
    }
}

__global__ __launch_bounds__(128) void k_trace_raster(const float *__restrict__ F, const int *__restrict__ node2x,
                                                      TabEntry *__restrict__ tab, float4 *__restrict__ exits,
                                                      RayParams p, unsigned long long *counters)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int e = blockIdx.y;
    const int N = p.N;
    const int nwarps = (N - 2 + 30) / 31;
    if (warp >= nwarps) return;  // whole warp leaves together
    const int j = 1 + 31 * warp + lane;      // this lane's ray
    const bool has_ray = j <= N - 1;
    TabEntry *fan = tab + (size_t)e * p.X;

    const double be = 2.0 * 3.14159265358979323846 * e / N;
    const float xe = (float)(p.R * cos(be)), ye = (float)(p.R * sin(be));
    const float gam0 = (float)(be + 3.14159265358979323846 / 2 + 3.14159265358979323846 * j / N);

    // reference and paraxial ray state
    float x = xe, y = ye, px, py, dxx = 0.f, dxy = 0.f, dpx, dpy, T = 0.f, Tc = 0.f;
    float J1 = 0.f, n1 = 0.f, Jlast = 0.f;
    int K = 0;
    {
        Fv f0;
        field_eval(F, p, x, y, f0);
        float s0, c0;
        sincosf(gam0, &s0, &c0);
        px = f0.n * c0; py = f0.n * s0;
        dpx = -f0.n * s0; dpy = f0.n * c0;
    }
    bool alive = has_ray;
    Vtx prev{}, nprev{};
    const float ds = p.ds;

    for (int i = 0; i < p.maxs; i++) {
        Vtx cur{};
        bool have = false;
        if (alive) {
            Fv F1, F2, F3;
            field_eval(F, p, x, y, F1);
            float n = F1.n;
            float pn = sqrtf(px * px + py * py);
            px *= n / pn; py *= n / pn;
            float qx = px / n, qy = py / n, qpx = F1.gx, qpy = F1.gy;
            float xa = x + ds * qx, ya = y + ds * qy;
            field_eval(F, p, xa, ya, F2);
            float pax = px + ds * qpx, pay = py + ds * qpy;
            float pan = sqrtf(pax * pax + pay * pay);
            pax *= F2.n / pan; pay *= F2.n / pan;
            float qax = pax / F2.n, qay = pay / F2.n, qpax = F2.gx, qpay = F2.gy;
            float sx = qx + qax, sy = qy + qay, sn = sqrtf(sx * sx + sy * sy);
            float dirx = sx / sn, diry = sy / sn;
            float xn = x + ds * dirx, yn = y + ds * diry;
            float pxn = px + ds * (qpx + qpax) * 0.5f, pyn = py + ds * (qpy + qpay) * 0.5f;
            // paraxial system, both stages at the reference ray's stage values
            float n2 = n * n;
            float gd = F1.gx * dxx + F1.gy * dxy, pd = px * dpx + py * dpy;
            float qdxx = -px * gd / n2 + dpx / n, qdxy = -py * gd / n2 + dpy / n;
            float qdpx = F1.hxx * dxx + F1.hxy * dxy - F1.gx * gd / n + F1.gx * pd / n2;
            float qdpy = F1.hxy * dxx + F1.hyy * dxy - F1.gy * gd / n + F1.gy * pd / n2;
            float dpax = dpx + ds * qdpx, dpay = dpy + ds * qdpy;
            float dxax = dxx + ds * qdxx, dxay = dxy + ds * qdxy;
            float na = F2.n, na2 = na * na;
            float gda = F2.gx * dxax + F2.gy * dxay, pda = pax * dpax + pay * dpay;
            float qdxax = -pax * gda / na2 + dpax / na, qdxay = -pay * gda / na2 + dpay / na;
            float qdpax = F2.hxx * dxax + F2.hxy * dxay - F2.gx * gda / na + F2.gx * pda / na2;
            float qdpay = F2.hxy * dxax + F2.hyy * dxay - F2.gy * gda / na + F2.gy * pda / na2;
            float dxxn = dxx + ds * (qdxx + qdxax) * 0.5f, dxyn = dxy + ds * (qdxy + qdxay) * 0.5f;
            float dpxn = dpx + ds * (qdpx + qdpax) * 0.5f, dpyn = dpy + ds * (qdpy + qdpay) * 0.5f;
            field_eval(F, p, xn, yn, F3);
            float inc = ds * (n + F3.n) * 0.5f;
            bool last = xn * xn + yn * yn >= p.R * p.R;
            if (last) {
                // final partial step: crossing of the step's chord with the ring; other
                // quantities interpolated linearly along the chord
                float b = x * dirx + y * diry, cc = x * x + y * y - p.R * p.R;
                float disc = b * b - cc;
                float t = -b + sqrtf(disc > 0.f ? disc : 0.f);
                t = fminf(fmaxf(t, 0.f), ds);
                float fr = t / ds;
                xn = x + t * dirx; yn = y + t * diry;
                inc *= fr;
                dxxn = dxx + fr * (dxxn - dxx); dxyn = dxy + fr * (dxyn - dxy);
                dpxn = dpx + fr * (dpxn - dpx); dpyn = dpy + fr * (dpyn - dpy);
                pxn = px + fr * (pxn - px); pyn = py + fr * (pyn - py);
                field_eval(F, p, xn, yn, F3);
            }
            // compensated travel-time sum (trapezoid of n along the samples)
            {
                float yk = inc - Tc, tk = T + yk;
                Tc = (tk - T) - yk;
                T = tk;
            }
            x = xn; y = yn; px = pxn; py = pyn; dxx = dxxn; dxy = dxyn; dpx = dpxn; dpy = dpyn;
            float pm = sqrtf(px * px + py * py), tx = px / pm, ty = py / pm;
            float J = dxx * ty - dxy * tx;
            if (i == 0) { J1 = J; n1 = F3.n; Jlast = J; }
            else if (J * Jlast < 0.f) K++;   // caustic: sign change of the ray Jacobian
            if (J != 0.f) Jlast = J;
            cur.x = x; cur.y = y; cur.T = T; cur.kx = tx; cur.ky = ty; cur.K = K;
            cur.a = sqrtf((n1 / F3.n) * fabsf(J1 / J) / ds);
            cur.id = j * 4096 + (i + 1);
            have = true;
            if (last) {
                alive = false;
                if (lane < 31 || j == N - 1)
                    exits[(size_t)e * (N - 1) + (j - 1)] = make_float4(atan2f(y, x), T, cur.a, (float)K);
            }
        }
        // neighbour ray j+1 (lane + 1): its sample i+1
        Vtx ncur;
        ncur.x = __shfl_down_sync(FULL, cur.x, 1);
        ncur.y = __shfl_down_sync(FULL, cur.y, 1);
        ncur.T = __shfl_down_sync(FULL, cur.T, 1);
        ncur.a = __shfl_down_sync(FULL, cur.a, 1);
        ncur.kx = __shfl_down_sync(FULL, cur.kx, 1);
        ncur.ky = __shfl_down_sync(FULL, cur.ky, 1);
        ncur.K = __shfl_down_sync(FULL, cur.K, 1);
        ncur.id = __shfl_down_sync(FULL, cur.id, 1);
        bool nhave = __shfl_down_sync(FULL, (int)have, 1) != 0;
        if (i >= 1 && have && nhave && lane < 31 && j + 1 <= N - 1) {
            uint32_t base = ((uint32_t)j << 11 | (uint32_t)i) << 1;   // 24-bit id, order (j, i, which)
            raster_tri(prev, nprev, ncur, base, p, node2x, fan, counters);
            raster_tri(prev, ncur, cur, base + 1, p, node2x, fan, counters);
        }
        prev = cur;
        nprev = ncur;
        if (!__any_sync(FULL, alive)) break;
        if (i == p.maxs - 1 && alive) atomicAdd(&counters[2], 1ull);   // ray never reached the ring
    }
}

void launch_trace_raster(const float *fields, const int *node2x, TabEntry *tab, float4 *exits, const RayParams &p,
                         unsigned long long *counters, cudaStream_t s)
{
    int nwarps = (p.N - 2 + 30) / 31;
    dim3 grd((nwarps + 3) / 4, p.N);
    k_trace_raster<<<grd, 128, 0, s>>>(fields, node2x, tab, exits, p, counters);
}

// ---------------------------------------------------------------- a4

__global__ void k_dgamma(const TabEntry *__restrict__ tab, float *__restrict__ dg, int N, int X,
                         unsigned long long *counters)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)N * X) return;
    int e = (int)(i / X), k = (int)(i % X);
    const TabEntry &tp = tab[(size_t)((e + 1) % N) * X + k];
    const TabEntry &tm = tab[(size_t)((e + N - 1) % N) * X + k];
    if (tab[i].idk == kUncovered) atomicAdd(&counters[0], 1ull);
    if (tp.idk == kUncovered || tm.idk == kUncovered) { dg[i] = 0.f; return; }
    float d = tp.gam - tm.gam;
    const float PI = 3.14159265358979f, TWO_PI = 6.28318530717959f;
    d = d - TWO_PI * floorf((d + PI) / TWO_PI);
    dg[i] = 0.5f * fabsf(d);
}

void launch_dgamma(const TabEntry *tab, float *dg, int N, int X, unsigned long long *counters, cudaStream_t s)
{
    size_t n = (size_t)N * X;
    k_dgamma<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tab, dg, N, X, counters);
}

// ---------------------------------------------------------------- a5

// Phase in cycles: f T - K/4 + 1/8, with f = fhi + flo and the product f T formed
// exactly enough (two-product) that omega T ~ 10^3 rad keeps ~1e-7 rad accuracy.
__device__ __forceinline__ float phase_cycles(float T, int K, float fhi, float flo)
{
    float p = fhi * T;
    float err = fmaf(fhi, T, -p) + flo * T;
    float r = (p - rintf(p)) + err;
    return r + 0.125f - 0.25f * (float)K;
}

__device__ __forceinline__ float wrap2pi(float t)
{
    const float TWO_PI = 6.28318530717959f;
    return t - TWO_PI * floorf(t / TWO_PI);
}

__global__ void k_direct_green(const float4 *__restrict__ exits, int N, float fhi, float flo, float C,
                               float2 *__restrict__ g, unsigned long long *counters)
{
    extern __shared__ float4 ex[];
    float *th = reinterpret_cast<float *>(ex + (N - 1));   // exit angle relative to beta_e, in [0, 2 pi)
    const int e = blockIdx.x;
    const double TWO_PI = 6.283185307179586476925;
    const double be = TWO_PI * e / N;
    for (int q = threadIdx.x; q < N - 1; q += blockDim.x) {
        float4 v = exits[(size_t)e * (N - 1) + q];
        ex[q] = v;
        double d = (double)v.x - be;
        th[q] = (float)(d - TWO_PI * floor(d / TWO_PI));
    }
    __syncthreads();
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
        if (r == e) { g[(size_t)e * N + r] = make_float2(0.f, 0.f); continue; }
        double td = TWO_PI * r / N - be;
        td -= TWO_PI * floor(td / TWO_PI);
        float t = (float)td;
        // first consecutive pair (j, j+1) whose exit angles bracket beta_r
        int found = -1;
        for (int j = 1; j <= N - 2; j++) {
            float tj = th[j - 1], tk = th[j];
            if (tj == tk) continue;
            if ((tj <= t && t <= tk) || (tk <= t && t <= tj)) { found = j; break; }
        }
        float T, a;
        int K;
        if (found > 0) {
            float4 A = ex[found - 1], B = ex[found];
            // the bracket fraction from the exit angles in double precision
            double ta = (double)A.x - be, tb = (double)B.x - be;
            ta -= TWO_PI * floor(ta / TWO_PI);
            tb -= TWO_PI * floor(tb / TWO_PI);
            double fr = (td - ta) / (tb - ta);
            T = (float)((double)A.y + fr * ((double)B.y - (double)A.y));
            a = (float)((double)A.z + fr * ((double)B.z - (double)A.z));
            K = (int)(fr < 0.5 ? A.w : B.w);
        } else {
            int best = 1;
            float bd = 1e30f;
            for (int j = 1; j <= N - 1; j++) {
                float d = fabsf(th[j - 1] - t);
                if (d < bd) { bd = d; best = j; }
            }
            float4 A = ex[best - 1];
            T = A.y; a = A.z; K = (int)A.w;
            atomicAdd(&counters[1], 1ull);
        }
        float sn, cs;
        sincospif(2.f * phase_cycles(T, K, fhi, flo), &sn, &cs);
        g[(size_t)e * N + r] = make_float2(C * a * cs, C * a * sn);
    }
}

void launch_direct_green(const float4 *exits, int N, double f, double c0, float2 *g, unsigned long long *counters,
                         cudaStream_t s)
{
    float fhi = (float)f, flo = (float)(f - (double)fhi);
    float C = (float)(1.0 / sqrt(8.0 * 3.14159265358979323846 * (2.0 * 3.14159265358979323846 * f) / c0));
    size_t smem = (size_t)(N - 1) * (sizeof(float4) + sizeof(float));   // <= 82 KB for N <= 4095
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_direct_green, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_direct_green<<<N, 256, smem, s>>>(exits, N, fhi, flo, C, g, counters);
}

// ---------------------------------------------------------------- table I/O

__global__ void k_set_tables(const float *T, const float *a, const float *gam, const uint8_t *K, TabEntry *tab,
                             size_t n)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    TabEntry t;
    float av = a[i];
    t.idk = av > 0.f ? (uint32_t)K[i] : kUncovered;
    t.T = T[i];
    t.a = av;
    t.gam = gam[i];
    tab[i] = t;
}

void launch_set_tables(const float *T, const float *a, const float *gam, const uint8_t *K, TabEntry *tab, size_t n,
                       cudaStream_t s)
{
    k_set_tables<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(T, a, gam, K, tab, n);
}

__global__ void k_get_tables(const TabEntry *tab, float *T, float *a, float *gam, uint8_t *K, size_t n)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    TabEntry t = tab[i];
    bool cov = t.idk != kUncovered;
    if (T) T[i] = cov ? t.T : 0.f;
    if (a) a[i] = cov ? t.a : 0.f;
    if (gam) gam[i] = cov ? t.gam : 0.f;
    if (K) K[i] = cov ? (uint8_t)(t.idk & 0xffu) : 0;
}

void launch_get_tables(const TabEntry *tab, float *T, float *a, float *gam, uint8_t *K, size_t n, cudaStream_t s)
{
    k_get_tables<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tab, T, a, gam, K, n);
}

}  // namespace rbx
