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
// lockstep; a block's four warps take the same rays of four neighbouring transducers. At
// each step a lane fetches its neighbour's new sample with a shuffle and rasterises the
// ray-tube quad (rays j, j+1; samples i, i+1) as two triangles straight
// into the fan's table (Sec. 4.4: triangulation of the ray samples). Overlapping triangles
// keep the first arrival: the 16-byte table entry starts with the key (T bits, triangle
// id, K) and a 128-bit compare-and-swap keeps the smallest key, so the table does not
// depend on the order in which warps finish. The ray samples are never stored.
//
// Fields are bilinearly interpolated from the field map (L1/L2 cached; a lossless trace on
// the smoothed map reads 24 B per node, 6 MB at 512^2). Travel time uses compensated (Kahan)
// summation.
#include <climits>

#include "rbx_internal.cuh"

namespace rbx {

// 1/v by the hardware approximation alone (within about 1 ulp): the Heun stages' 1/n, which
// scales the direction and the paraxial terms; the refined rcp_nr serves the rest.
__device__ __forceinline__ float rcp_ap(float v)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ int clampi_(int i, int lo, int hi) { return i < lo ? lo : (i > hi ? hi : i); }

struct Fv {
    float n, gx, gy, hxx, hxy, hyy, al;   // al: absorption coefficient alpha (lossy media only)
    float nr;                              // slowness integrated along the ray (n, or the non-smoothed one)
};

// s += inc with compensation term c (Kahan): the ray state is a sum of ~10^3 small steps
__device__ __forceinline__ void kadd(float &s, float &c, float inc)
{
    const float y = inc - c, t = s + y;
    c = (t - s) - y;
    s = t;
}

template <bool LOSSY, bool RAW>
__device__ __forceinline__ void field_eval(const float *__restrict__ F, const RayParams &p, float px, float py, Fv &o)
{
    float u = (px - p.x0) * p.inv_dx, v = (py - p.y0) * p.inv_dx;
    int i = clampi_((int)floorf(u), 0, p.nx - 2), j = clampi_((int)floorf(v), 0, p.ny - 2);
    float tx = u - (float)i, ty = v - (float)j;
    const size_t nxy = (size_t)p.nx * p.ny, k00 = (size_t)j * p.nx + i, k01 = k00 + p.nx;
    const float4 *F4 = reinterpret_cast<const float4 *>(F);
    const float2 *F2 = reinterpret_cast<const float2 *>(F4 + nxy);
    float4 a0 = __ldg(F4 + k00), b0 = __ldg(F4 + k00 + 1), c0 = __ldg(F4 + k01), d0 = __ldg(F4 + k01 + 1);
    float2 a1 = __ldg(F2 + k00), b1 = __ldg(F2 + k00 + 1), c1 = __ldg(F2 + k01), d1 = __ldg(F2 + k01 + 1);
    float w00 = (1.f - tx) * (1.f - ty), w10 = tx * (1.f - ty), w01 = (1.f - tx) * ty, w11 = tx * ty;
    o.n = w00 * a0.x + w10 * b0.x + w01 * c0.x + w11 * d0.x;
    o.gx = w00 * a0.y + w10 * b0.y + w01 * c0.y + w11 * d0.y;
    o.gy = w00 * a0.z + w10 * b0.z + w01 * c0.z + w11 * d0.z;
    o.hxx = w00 * a0.w + w10 * b0.w + w01 * c0.w + w11 * d0.w;
    o.hxy = w00 * a1.x + w10 * b1.x + w01 * c1.x + w11 * d1.x;
    o.hyy = w00 * a1.y + w10 * b1.y + w01 * c1.y + w11 * d1.y;
    if (LOSSY || RAW) {
        const float2 *F3 = F2 + nxy;
        float2 a2 = __ldg(F3 + k00), b2 = __ldg(F3 + k00 + 1), c2 = __ldg(F3 + k01), d2 = __ldg(F3 + k01 + 1);
        o.al = LOSSY ? w00 * a2.x + w10 * b2.x + w01 * c2.x + w11 * d2.x : 0.f;
        o.nr = RAW ? w00 * a2.y + w10 * b2.y + w01 * c2.y + w11 * d2.y : o.n;
    } else {
        o.al = 0.f;
        o.nr = o.n;
    }
}

// A ray sample as a triangle vertex.
struct Vtx {
    float x, y, T, a, kx, ky;
    int K;
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

// Keep the entry with the smaller key, starting from a known content (lo, hi) of the
// entry. Every successful exchange lowers the stored key, so the loop ends after at most as
// many rounds as there are competing triangles (the bound only reports a broken invariant).
__device__ __forceinline__ void cas_min_from(TabEntry *e, unsigned long long key, unsigned long long pay,
                                             unsigned long long lo, unsigned long long hi,
                                             unsigned long long *counters)
{
    unsigned long long *a = reinterpret_cast<unsigned long long *>(e);
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

// Per-warp queue of table hits in shared memory, drained 32 at a time (one per lane):
// node, key, and the interpolated amplitude and direction (the direction angle is formed
// at the drain, where all 32 lanes are busy).
struct HitQueue {
    int *xi;
    unsigned long long *key;
    float4 *v;       // (a, kappa_x, kappa_y, -)
    unsigned *cov;   // entries this warp found untouched (each entry is found so exactly once)
    int n;           // warp-uniform
};

// Returns true when this exchange was the entry's first write.
__device__ __forceinline__ bool drain_one(const HitQueue &hq, int q, TabEntry *fan, unsigned long long *counters)
{
    const float4 v = hq.v[q];
    const unsigned long long key = hq.key[q];
    const unsigned long long pay = ((unsigned long long)__float_as_uint(atan2f(v.z, v.y)) << 32) | __float_as_uint(v.x);
    TabEntry *addr = fan + hq.xi[q];
    // most entries are still untouched (all ones): try that first, then take the minimum
    unsigned long long lo, hi;
    cas128(reinterpret_cast<unsigned long long *>(addr), ~0ull, ~0ull, key, pay, lo, hi);
    if (lo == ~0ull && hi == ~0ull) return true;
    cas_min_from(addr, key, pay, lo, hi, counters);
    return false;
}

// Adds the warp's first writes to its count of covered entries (all lanes take part).
__device__ __forceinline__ void count_first(const HitQueue &hq, bool first)
{
    const unsigned b = __ballot_sync(0xffffffffu, first);
    if ((threadIdx.x & 31) == 0) *hq.cov += __popc(b);
}

// Edge function of P -> Q at (px, py), always evaluated from the vertex with the smaller
// id (ids order P[j,i] < P[j,i+1] < P[j+1,i] < P[j+1,i+1]), so the triangles on both sides
// of an edge see exactly opposite values and no node falls between them.
__device__ __forceinline__ float edge_fn(const Vtx &P, const Vtx &Q, float px, float py)
{
    return __fmaf_rn(Q.x - P.x, py - P.y, -__fmul_rn(Q.y - P.y, px - P.x));
}

__device__ __forceinline__ bool tri_inside(float eA, float eB, float eC, float &sum)
{
    sum = eA + eB + eC;
    bool in = sum > 0.f ? (eA >= 0.f && eB >= 0.f && eC >= 0.f) : (eA <= 0.f && eB <= 0.f && eC <= 0.f);
    return in && sum != 0.f;
}

__device__ __forceinline__ unsigned long long tri_key(const Vtx &A, const Vtx &B, const Vtx &C, float lb, float lc,
                                                      uint32_t tid)
{
    float T = A.T + lb * (B.T - A.T) + lc * (C.T - A.T);
    int K = max(A.K, max(B.K, C.K));
    return ((unsigned long long)__float_as_uint(T) << 32) | ((unsigned long long)tid << 8) |
           (unsigned long long)min(K, 255);
}

// Rasterise the ray-tube quad P00 = P[j,i], P01 = P[j,i+1], P10 = P[j+1,i], P11 = P[j+1,i+1]
// of every valid lane as triangles t0 = (P00, P10, P11) and t1 = (P00, P11, P01) (ids
// tid0, tid0 + 1). Called by the whole warp. A node inside both triangles (on the shared
// diagonal) keeps the smaller key locally; hits go to the warp's queue. rows[iy] gives the
// mask nodes of grid row iy: (first compact index, first ix, last ix).
__device__ __forceinline__ void raster_quad_warp(bool valid, const Vtx &P00, const Vtx &P01, const Vtx &P10,
                                                 const Vtx &P11, uint32_t tid0, const RayParams &p, float inv_dx,
                                                 const int4 *rows, TabEntry *fan, HitQueue &hq,
                                                 unsigned long long *counters)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    bool ok0 = false, ok1 = false;
    float ar0 = 0.f, ar1 = 0.f;
    int ix0 = 0, iy0 = 0, w = 0, cnt = 0;
    if (valid) {
        const float tiny = 1e-9f * p.ds * p.ds;
        ar0 = (P10.x - P00.x) * (P11.y - P00.y) - (P10.y - P00.y) * (P11.x - P00.x);
        ar1 = (P11.x - P00.x) * (P01.y - P00.y) - (P11.y - P00.y) * (P01.x - P00.x);
        ok0 = fabsf(ar0) > tiny;
        ok1 = fabsf(ar1) > tiny;
        if (ok0 || ok1) {
            float minx = fminf(fminf(P00.x, P01.x), fminf(P10.x, P11.x));
            float maxx = fmaxf(fmaxf(P00.x, P01.x), fmaxf(P10.x, P11.x));
            float miny = fminf(fminf(P00.y, P01.y), fminf(P10.y, P11.y));
            float maxy = fmaxf(fmaxf(P00.y, P01.y), fmaxf(P10.y, P11.y));
            // candidate nodes of the bounding box, widened by 1e-3 cells: in FP32 the box's grid
            // coordinates carry ~2e-5 cells of rounding, and a node that lies on a box edge (at a
            // triangle's tip) must stay a candidate of every quad that may hold it; the edge
            // functions below decide which does
            const float slack = 1e-3f;
            ix0 = max(0, (int)ceilf((minx - p.x0) * inv_dx - slack));
            int ix1 = min(p.nx - 1, (int)floorf((maxx - p.x0) * inv_dx + slack));
            iy0 = max(0, (int)ceilf((miny - p.y0) * inv_dx - slack));
            int iy1 = min(p.ny - 1, (int)floorf((maxy - p.y0) * inv_dx + slack));
            w = ix1 - ix0 + 1;
            int h = iy1 - iy0 + 1;
            cnt = (w > 0 && h > 0) ? w * h : 0;
        }
    }
    // A folded quad (its triangles of opposite orientation) can hold a node in both
    // triangles; otherwise only the triangle on the node's side of the diagonal P00-P11 can.
    const bool fold = ok0 && ok1 && ((ar0 > 0.f) != (ar1 > 0.f));
    int ix = ix0, iy = iy0;
    for (int it = 0; __any_sync(FULL, it < cnt); it++) {
        bool act = false, hit = false;
        int xi = 0;
        float px = 0.f, py = 0.f, e3 = 0.f;
        if (it < cnt) {
            const int4 ro = rows[iy];
            if (ix >= ro.y && ix <= ro.z) {
                act = true;
                xi = ro.x + ix - ro.y;
                px = p.x0 + (float)ix * p.dx;
                py = p.y0 + (float)iy * p.dx;
                e3 = edge_fn(P00, P11, px, py);
            }
            if (++ix >= ix0 + w) { ix = ix0; iy++; }
        }
        unsigned long long key = ~0ull;
        float4 hv = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool both = act && ok0 && ok1 && (fold || e3 == 0.f);
        if (__any_sync(FULL, both)) {
            // both triangles, the smaller key wins (nodes on the diagonal, folded quads)
            if (act) {
                const float e1 = edge_fn(P00, P10, px, py), e2 = edge_fn(P10, P11, px, py);
                const float e4 = edge_fn(P01, P11, px, py), e5 = edge_fn(P00, P01, px, py);
                float s0, s1, lb0 = 0.f, lc0 = 0.f, lb1 = 0.f, lc1 = 0.f;
                unsigned long long k0 = ~0ull, k1 = ~0ull;
                if (ok0 && tri_inside(e2, -e3, e1, s0)) {
                    float inv = rcp_nr(s0);
                    lb0 = -e3 * inv;
                    lc0 = e1 * inv;
                    k0 = tri_key(P00, P10, P11, lb0, lc0, tid0);
                }
                if (ok1 && tri_inside(-e4, -e5, e3, s1)) {
                    float inv = rcp_nr(s1);
                    lb1 = -e5 * inv;
                    lc1 = e3 * inv;
                    k1 = tri_key(P00, P11, P01, lb1, lc1, tid0 + 1);
                }
                if (k0 != ~0ull || k1 != ~0ull) {
                    const bool use0 = k0 < k1;
                    const float lb = use0 ? lb0 : lb1, lc = use0 ? lc0 : lc1, la = 1.f - lb - lc;
                    const float Ba = use0 ? P10.a : P11.a, Ca = use0 ? P11.a : P01.a;
                    const float Bkx = use0 ? P10.kx : P11.kx, Ckx = use0 ? P11.kx : P01.kx;
                    const float Bky = use0 ? P10.ky : P11.ky, Cky = use0 ? P11.ky : P01.ky;
                    hv = make_float4(la * P00.a + lb * Ba + lc * Ca, la * P00.kx + lb * Bkx + lc * Ckx,
                                     la * P00.ky + lb * Bky + lc * Cky, 0.f);
                    key = use0 ? k0 : k1;
                    hit = true;
                }
            }
        } else if (act) {
            // one triangle: t1 = (P00, P11, P01) where e3 has t1's orientation, else
            // t0 = (P00, P10, P11). With M = P01 (t1) or P10 (t0) its other edges are M -> P11
            // and P00 -> M, evaluated exactly as in the two-triangle path.
            const bool use1 = ok1 && (!ok0 || ((e3 > 0.f) == (ar1 > 0.f)));
            const Vtx &M = use1 ? P01 : P10;
            const float x1 = edge_fn(M, P11, px, py), x2 = edge_fn(P00, M, px, py);
            const float eBC = use1 ? -x1 : x1, eCA = use1 ? -x2 : -e3, eAB = use1 ? e3 : x2;
            float s;
            if (tri_inside(eBC, eCA, eAB, s)) {
                const float inv = rcp_nr(s), lb = eCA * inv, lc = eAB * inv, la = 1.f - lb - lc;
                const Vtx &B = use1 ? P11 : P10, &C = use1 ? P01 : P11;
                key = tri_key(P00, B, C, lb, lc, tid0 + (use1 ? 1u : 0u));
                hv = make_float4(la * P00.a + lb * B.a + lc * C.a, la * P00.kx + lb * B.kx + lc * C.kx,
                                 la * P00.ky + lb * B.ky + lc * C.ky, 0.f);
                hit = true;
            }
        }
        const unsigned b = __ballot_sync(FULL, hit);
        if (b) {
            const int slot = hq.n + __popc(b & ((1u << lane) - 1));
            if (hit) {
                hq.xi[slot] = xi;
                hq.key[slot] = key;
                hq.v[slot] = hv;
            }
            hq.n += __popc(b);
            __syncwarp();
            if (hq.n >= 32) {
                count_first(hq, drain_one(hq, hq.n - 32 + lane, fan, counters));
                hq.n -= 32;
                __syncwarp();
            }
        }
    }
}

// Warps per block, each tracing the same rays of a neighbouring transducer; 20 warps per SM.
constexpr int kFansPerBlock = 4;

// The per-warp hit queues of a block (shared memory).
struct BlockQueues {
    int xi[kFansPerBlock][64];
    unsigned long long key[kFansPerBlock][64];
    float4 v[kFansPerBlock][64];
    unsigned cov[kFansPerBlock];
};

// One block's work: warp `warp` of the fans of fan block `eblk` (fans 4 eblk .. 4 eblk + 3),
// one warp per fan; `rows` (the mask's row ranges) and the queues' coverage counts are set up
// by the caller. No block-wide barrier inside: a warp may return early.
template <bool LOSSY, bool RAW>
__device__ __forceinline__ void trace_block(const float *__restrict__ F, const int4 *rows, TabEntry *__restrict__ tab,
                                            float4 *__restrict__ exits, const RayParams &p,
                                            unsigned long long *counters, int warp, int eblk, BlockQueues &bq)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    // the warps of a block trace the same 32 rays of neighbouring transducers: rotated by one
    // ring step, those rays stay within about a cell of one another, so their field gathers
    // share L1 lines
    const int e = eblk * kFansPerBlock + wib;
    const int N = p.N;
    const int nwarps = (N - 2 + 30) / 31;
    if (warp >= nwarps || e >= N) return;  // whole warp leaves together
    const int j = 1 + 31 * warp + lane;      // this lane's ray
    const bool has_ray = j <= N - 1;
    TabEntry *fan = tab + (size_t)e * p.X;
    const float ds = p.ds, hds = 0.5f * p.ds, inv_dx = p.inv_dx, R2 = p.R * p.R;
    HitQueue hq{bq.xi[wib], bq.key[wib], bq.v[wib], &bq.cov[wib], 0};

    const double be = p.beta ? p.beta[e] : 2.0 * 3.14159265358979323846 * e / N;
    float x = (float)(p.R * cos(be)), y = (float)(p.R * sin(be));
    const float gam0 = (float)(be + 3.14159265358979323846 / 2 + 3.14159265358979323846 * j / N);

    // reference ray (x, p) and paraxial ray (dx, dp); F1 caches the fields at x
    Fv F1;
    field_eval<LOSSY, RAW>(F, p, x, y, F1);
    float px, py, dpx, dpy, dxx = 0.f, dxy = 0.f, T = 0.f, Tc = 0.f;
    float B = 0.f, Bc = 0.f;   // lossy media: B = int alpha ds by the rule of T; a gains exp(-B)
    // compensation terms of the position and of the paraxial ray's closed-form steps (T has
    // Tc). In the Heun steps the momentum, renormalised to n(x) at every step, and the
    // paraxial ray, which only sets the amplitude, take plain sums: compensated too, the
    // tables met the same parity bars against the FP64 oracle (T 1e-9 s, a 1e-5) and the
    // trace took 1.6 % longer.
    float cx = 0.f, cy = 0.f, cdx = 0.f, cdy = 0.f;

    // Uniform water near the ring (exact up to rounding). Beyond radius rho every cell that a
    // sample or an auxiliary point can touch holds the same medium with zero derivatives (rho
    // exceeds the largest radius of a non-uniform node by a cell diagonal and a step), so there
    // a ray is a straight line with constant n and a linearly growing paraxial deviation; rho
    // also stays two cells outside the mask, so a quad with all vertices beyond rho holds no
    // mask node. Up to its entry step kin (its last sample beyond rho on the way in) a ray
    // takes the closed form of the step; kin depends on the ray alone, so the ray shared by two
    // warps has identical samples in both. The warp rasterises nothing before its smallest kin.
    const float ru = __uint_as_float((unsigned)counters[7]);
    const float rho = fmaxf(ru + 1.5f * p.dx + ds, p.rmask + 2.f * p.dx), rho2 = rho * rho;
    int kin = 0;
    {
        float s0, c0;
        sincosf(gam0, &s0, &c0);
        px = F1.n * c0; py = F1.n * s0;
        dpx = -F1.n * s0; dpy = F1.n * c0;
        if (has_ray && R2 > rho2) {
            const float b = x * c0 + y * s0, disc = b * b - (fmaf(x, x, y * y) - rho2);
            const float s_in = disc >= 0.f ? -b - sqrtf(disc) : -b;   // entry, or closest approach
            kin = max(0, (int)floorf(s_in / ds) - 1);
        }
    }
    const int i0 = __reduce_min_sync(FULL, has_ray ? kin : 0x7fffffff);
    const float rm = p.rmask + 2.f * p.dx, rm2 = rm * rm;
    float sc1 = 0.f, Jlast = 0.f;   // sc1 = sqrt(n_1 |J_1| / ds): a_i = sc1 / sqrt(n_i |J_i|)
    int K = 0;
    bool alive = has_ray;
    Vtx prev{}, nprev{};

    for (int i = 0; i < p.maxs; i++) {
        Vtx cur{};
        bool have = false;
        if (alive && i < kin) {
            // the step below in a uniform medium: straight, p constant, dx += ds dp / n
            const float n = F1.n, in = rcp_nr(n);
            const float rp = rsqrtf(px * px + py * py), tx = px * rp, ty = py * rp;
            kadd(x, cx, ds * tx); kadd(y, cy, ds * ty);
            kadd(dxx, cdx, ds * (dpx * in)); kadd(dxy, cdy, ds * (dpy * in));
            kadd(T, Tc, hds * (F1.nr + F1.nr));
            if (LOSSY) kadd(B, Bc, hds * (F1.al + F1.al));
            const float J = dxx * ty - dxy * tx;
            if (i == 0) { sc1 = sqrtf(F1.nr * fabsf(J) / ds); Jlast = J; }
            else if (J * Jlast < 0.f) K++;
            if (J != 0.f) Jlast = J;
            cur.x = x; cur.y = y; cur.T = T; cur.kx = tx; cur.ky = ty; cur.K = K;
            cur.a = sc1 * rsqrtf(F1.nr * fabsf(J));
            if (LOSSY) cur.a *= expf(-B);
            have = true;
        } else if (alive) {
            // stage 1 at x: normalise p to n(x), q_x = p/n, q_p = grad n
            const float n = F1.n, in = rcp_ap(n);
            const float sc = n * rsqrtf(px * px + py * py);
            px *= sc; py *= sc;
            const float qx = px * in, qy = py * in;
            // stage 2 at the auxiliary point x + ds q_x
            Fv F2;
            field_eval<LOSSY, RAW>(F, p, x + ds * qx, y + ds * qy, F2);
            const float na = F2.n, ina = rcp_ap(na);
            float pax = px + ds * F1.gx, pay = py + ds * F1.gy;
            const float sca = na * rsqrtf(pax * pax + pay * pay);
            pax *= sca; pay *= sca;
            const float qax = pax * ina, qay = pay * ina;
            const float sx = qx + qax, sy = qy + qay, rs = rsqrtf(sx * sx + sy * sy);
            const float dirx = sx * rs, diry = sy * rs;
            const float ddpx = hds * (F1.gx + F2.gx), ddpy = hds * (F1.gy + F2.gy);
            // paraxial system, both stages at the reference ray's stage values:
            // q_dx = (dp - p (g.dx)/n)/n, q_dp = H dx + g ((p.dp)/n - g.dx)/n
            const float gd = F1.gx * dxx + F1.gy * dxy, pd = px * dpx + py * dpy;
            const float qdxx = in * (dpx - px * gd * in), qdxy = in * (dpy - py * gd * in);
            const float w1 = in * (pd * in - gd);
            const float qdpx = F1.hxx * dxx + F1.hxy * dxy + F1.gx * w1;
            const float qdpy = F1.hxy * dxx + F1.hyy * dxy + F1.gy * w1;
            const float dpax = dpx + ds * qdpx, dpay = dpy + ds * qdpy;
            const float dxax = dxx + ds * qdxx, dxay = dxy + ds * qdxy;
            const float gda = F2.gx * dxax + F2.gy * dxay, pda = pax * dpax + pay * dpay;
            const float qdxax = ina * (dpax - pax * gda * ina), qdxay = ina * (dpay - pay * gda * ina);
            const float w2 = ina * (pda * ina - gda);
            const float qdpax = F2.hxx * dxax + F2.hxy * dxay + F2.gx * w2;
            const float qdpay = F2.hxy * dxax + F2.hyy * dxay + F2.gy * w2;
            const float ddxx = hds * (qdxx + qdxax), ddxy = hds * (qdxy + qdxay);
            const float ddpx2 = hds * (qdpx + qdpax), ddpy2 = hds * (qdpy + qdpay);
            const float xn = x + ds * dirx, yn = y + ds * diry;
            field_eval<LOSSY, RAW>(F, p, xn, yn, F2);                // fields at the new sample (reused next step)
            float inc = hds * (F1.nr + F2.nr), incB = LOSSY ? hds * (F1.al + F2.al) : 0.f;
            const bool last = xn * xn + yn * yn >= R2;
            if (last) {
                // final partial step: crossing of the step's chord with the ring; the other
                // quantities interpolated linearly along the chord. A first step starts at the
                // transducer, on the ring: |x|^2 - R^2 is 0 there, and its FP32 rounding residue
                // (~R ulp(R)) would swamp b^2 for the near-tangent rays that end within a step
                float b = x * dirx + y * diry, cc = i == 0 ? 0.f : x * x + y * y - R2;
                float disc = b * b - cc;
                float t = -b + sqrtf(disc > 0.f ? disc : 0.f);
                t = fminf(fmaxf(t, 0.f), ds);
                float fr = t / ds;
                x = x + t * dirx; y = y + t * diry;
                inc *= fr;
                incB *= fr;
                dxx += fr * ddxx; dxy += fr * ddxy;
                dpx += fr * ddpx2; dpy += fr * ddpy2;
                px += fr * ddpx; py += fr * ddpy;
                field_eval<LOSSY, RAW>(F, p, x, y, F2);
            } else {
                kadd(x, cx, ds * dirx); kadd(y, cy, ds * diry);
                px += ddpx; py += ddpy;
                dxx += ddxx; dxy += ddxy;
                dpx += ddpx2; dpy += ddpy2;
            }
            kadd(T, Tc, inc);   // trapezoid of n along the samples
            if (LOSSY) kadd(B, Bc, incB);
            F1 = F2;
            const float rp = rsqrtf(px * px + py * py), tx = px * rp, ty = py * rp;
            const float J = dxx * ty - dxy * tx;
            if (i == 0) { sc1 = sqrtf(F1.nr * fabsf(J) / ds); Jlast = J; }
            else if (J * Jlast < 0.f) K++;   // caustic: sign change of the ray Jacobian
            if (J != 0.f) Jlast = J;
            cur.x = x; cur.y = y; cur.T = T; cur.kx = tx; cur.ky = ty; cur.K = K;
            cur.a = sc1 * rsqrtf(F1.nr * fabsf(J));
            if (LOSSY) cur.a *= expf(-B);
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
        const bool nhave = __shfl_down_sync(FULL, (int)have, 1) != 0;
        const bool valid = i >= 1 && i >= i0 && have && nhave && lane < 31 && j + 1 <= N - 1;
        // A quad beyond a line two cells outside the mask holds no mask node, in any medium:
        // the edge functions accept only points of its two triangles, which lie in the convex
        // hull of its corners, so when every corner q has u.q > rm for u the direction of the
        // corners' sum, so does every accepted point, and |q| > rm. The warp skips the step's
        // rasterisation when that holds for all its quads. The corners' own radii beyond rm
        // are necessary for it and cheap, so the line test runs only when they hold for the
        // whole warp (radii alone would not do: the cross edge of a wide tube can be a chord
        // through the mask).
        const bool ob = fmaf(cur.x, cur.x, cur.y * cur.y) > rm2 && fmaf(prev.x, prev.x, prev.y * prev.y) > rm2;
        const bool nb = __shfl_down_sync(FULL, (int)ob, 1) != 0;
        bool skip = __all_sync(FULL, !valid || (ob && nb));
        if (skip) {
            bool hs = true;
            if (valid) {
                const float gx = (prev.x + cur.x) + (nprev.x + ncur.x), gy = (prev.y + cur.y) + (nprev.y + ncur.y);
                const float h = fminf(fminf(fmaf(gx, prev.x, gy * prev.y), fmaf(gx, cur.x, gy * cur.y)),
                                      fminf(fmaf(gx, nprev.x, gy * nprev.y), fmaf(gx, ncur.x, gy * ncur.y)));
                hs = h > 0.f && h * h > rm2 * fmaf(gx, gx, gy * gy);
            }
            skip = __all_sync(FULL, hs);
        }
        if (!skip)
            raster_quad_warp(valid, prev, cur, nprev, ncur, ((uint32_t)j << 11 | (uint32_t)i) << 1, p, inv_dx, rows,
                             fan, hq, counters);
        prev = cur;
        nprev = ncur;
        // Leaving through the uniform water: once a ray is beyond rho, moving outward, and so
        // are (or have ended) the rays it forms quads with in this warp, no later quad of it
        // can hold a mask node, and it goes straight to the ring in closed form (the chord's
        // crossing as in the last step above; J is linear in s there, so at most one caustic).
        {
            const bool out = alive && i >= kin && fmaf(x, x, y * y) > rho2 && fmaf(x, px, y * py) > 0.f;
            if (__any_sync(FULL, out)) {
                const bool okself = !alive || out;
                bool okL = __shfl_up_sync(FULL, okself, 1), okR = __shfl_down_sync(FULL, okself, 1);
                const bool aL = __shfl_up_sync(FULL, alive, 1), aR = __shfl_down_sync(FULL, alive, 1);
                const float xl = __shfl_up_sync(FULL, x, 1), yl = __shfl_up_sync(FULL, y, 1);
                const float xr = __shfl_down_sync(FULL, x, 1), yr = __shfl_down_sync(FULL, y, 1);
                const float gap = rho - p.rmask, gap2 = gap * gap;
                if (lane == 0) okL = true;
                else if (aL) okL = okL && (x - xl) * (x - xl) + (y - yl) * (y - yl) < gap2;
                if (lane == 31) okR = true;
                else if (aR) okR = okR && (x - xr) * (x - xr) + (y - yr) * (y - yr) < gap2;
                if (out && okL && okR) {
                    const float n = F1.n, in = rcp_nr(n), inc = hds * (F1.nr + F1.nr);
                    const float rp = rsqrtf(px * px + py * py), tx = px * rp, ty = py * rp;
                    const float b = x * tx + y * ty, se = -b + sqrtf(fmaxf(b * b - (fmaf(x, x, y * y) - R2), 0.f));
                    const int m = max(0, (int)floorf(se / ds));
                    const float sm = (float)m * ds;
                    const float xm = fmaf(sm, tx, x), ym = fmaf(sm, ty, y);
                    const float b2 = xm * tx + ym * ty, disc = b2 * b2 - (fmaf(xm, xm, ym * ym) - R2);
                    float t = -b2 + sqrtf(disc > 0.f ? disc : 0.f);
                    t = fminf(fmaxf(t, 0.f), ds);
                    x = fmaf(t, tx, xm); y = fmaf(t, ty, ym);
                    kadd(T, Tc, (float)m * inc);
                    kadd(T, Tc, (t / ds) * inc);
                    if (LOSSY) {
                        const float incB = hds * (F1.al + F1.al);
                        kadd(B, Bc, (float)m * incB);
                        kadd(B, Bc, (t / ds) * incB);
                    }
                    dxx = fmaf(sm + t, dpx * in, dxx); dxy = fmaf(sm + t, dpy * in, dxy);
                    field_eval<LOSSY, RAW>(F, p, x, y, F1);
                    const float J = dxx * ty - dxy * tx;
                    if (J * Jlast < 0.f) K++;
                    const float a = sc1 * rsqrtf(F1.nr * fabsf(J)) * (LOSSY ? expf(-B) : 1.f);
                    if (lane < 31 || j == N - 1)
                        exits[(size_t)e * (N - 1) + (j - 1)] = make_float4(atan2f(y, x), T, a, (float)K);
                    alive = false;
                }
            }
        }
        if (!__any_sync(FULL, alive)) break;
        if (i == p.maxs - 1 && alive) atomicAdd(&counters[2], 1ull);   // ray never reached the ring
    }
    // drain the rest of the queue; the covered-entry count goes to counters[0]
    count_first(hq, lane < hq.n && drain_one(hq, lane, fan, counters));
    __syncwarp();
    if (lane == 0 && *hq.cov) atomicAdd(&counters[0], (unsigned long long)*hq.cov);
}

template <bool LOSSY, bool RAW>
__global__ __launch_bounds__(32 * kFansPerBlock, 20 / kFansPerBlock) void k_trace_raster(const float *__restrict__ F, const int4 *__restrict__ rows_g,
                                                         TabEntry *__restrict__ tab, float4 *__restrict__ exits,
                                                         RayParams p, unsigned long long *counters)
{
    extern __shared__ int4 rows[];                          // [ny] mask row ranges
    __shared__ BlockQueues bq;
    for (int q = threadIdx.x; q < p.ny; q += blockDim.x) rows[q] = rows_g[q];
    if (threadIdx.x < kFansPerBlock) bq.cov[threadIdx.x] = 0u;
    __syncthreads();
    trace_block<LOSSY, RAW>(F, rows, tab, exits, p, counters, blockIdx.x, blockIdx.y, bq);
}

// Persistent form of the trace over several jobs (the batched form). Each block takes the
// next item from a device counter until the list is exhausted: items are numbered job by job
// in the order of g.j, and within a job as the blocks of the per-job grid (warps fastest). An
// item is one block of the per-job kernel. The job list is a kernel parameter, so that the
// jobs' parameters stay in the constant bank (with them in shared memory the kernel spilled
// and ran 5.8 % slower per item; this form costs 1.1 %).
template <bool LOSSY, bool RAW>
__global__ __launch_bounds__(32 * kFansPerBlock, 20 / kFansPerBlock) void k_trace_grouped(const __grid_constant__ TraceGroup g,
                                                                                        int *next)
{
    extern __shared__ int4 rows[];   // [largest ny of the jobs]
    __shared__ BlockQueues bq;
    __shared__ int s_item, s_job;
    for (;;) {
        __syncthreads();   // the block's warps are done with the previous item
        if (threadIdx.x == 0) {
            const int it = atomicAdd(next, 1);
            int jb = 0;
            if (it < g.total)
                while (jb + 1 < g.njobs && g.j[jb + 1].item0 <= it) jb++;
            s_item = it;
            s_job = jb;
        }
        __syncthreads();
        const int it = s_item;
        if (it >= g.total) return;   // uniform over the block
        const TraceJob &J = g.j[s_job];
        for (int q = threadIdx.x; q < J.p.ny; q += blockDim.x) rows[q] = J.rows[q];
        if (threadIdx.x < kFansPerBlock) bq.cov[threadIdx.x] = 0u;
        __syncthreads();
        const int local = it - J.item0;
        trace_block<LOSSY, RAW>(J.F, rows, J.tab, J.exits, J.p, J.counters, local % J.nwarps, local / J.nwarps, bq);
    }
}

// Largest radius of a node whose fields differ from the uniform medium of node (0, 0)
// (n, alpha and the integrated slowness there, all derivatives zero); +inf when node (0, 0)
// itself is not uniform.
__global__ void k_uniform_radius(const float4 *__restrict__ F, RayParams p, unsigned long long *ru)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned r = 0u;   // bits of a non-negative float: their order is the values' order
    if (k < p.nx * p.ny) {
        const size_t nxy = (size_t)p.nx * p.ny;
        const float2 *F2 = reinterpret_cast<const float2 *>(F + nxy), *F3 = F2 + nxy;
        const float4 u0 = F[0], a0 = F[k];
        const float2 v0 = F2[0], v1 = F3[0], b0 = F2[k], b1 = F3[k];
        const float4 u1 = make_float4(v0.x, v0.y, v1.x, v1.y), a1 = make_float4(b0.x, b0.y, b1.x, b1.y);
        if (k == 0 && !(u0.y == 0.f && u0.z == 0.f && u0.w == 0.f && u1.x == 0.f && u1.y == 0.f)) {
            r = 0x7f800000u;   // +inf
        } else {
            const bool uni = a0.x == u0.x && a0.y == 0.f && a0.z == 0.f && a0.w == 0.f && a1.x == 0.f &&
                             a1.y == 0.f && a1.z == u1.z && a1.w == u1.w;
            if (!uni) {
                const float px = p.x0 + (float)(k % p.nx) * p.dx, py = p.y0 + (float)(k / p.nx) * p.dx;
                r = __float_as_uint(sqrtf(px * px + py * py));
            }
        }
    }
    r = __reduce_max_sync(0xffffffffu, r);   // one atomic per warp
    if ((threadIdx.x & 31) == 0 && r) atomicMax(ru, (unsigned long long)r);
}

void launch_uniform_radius(const float *fields, const RayParams &p, unsigned long long *ru, cudaStream_t s)
{
    const int n = p.nx * p.ny;
    k_uniform_radius<<<(n + 255) / 256, 256, 0, s>>>(reinterpret_cast<const float4 *>(fields), p, ru);
}

void launch_trace_raster(const float *fields, const int4 *rows, TabEntry *tab, float4 *exits, const RayParams &p,
                         unsigned long long *counters, bool lossy, bool raw, cudaStream_t s)
{
    int nwarps = (p.N - 2 + 30) / 31;
    dim3 grd(nwarps, (p.N + kFansPerBlock - 1) / kFansPerBlock);
    const size_t sm = (size_t)p.ny * sizeof(int4);
    if (lossy && raw)
        k_trace_raster<true, true><<<grd, 32 * kFansPerBlock, sm, s>>>(fields, rows, tab, exits, p, counters);
    else if (lossy)
        k_trace_raster<true, false><<<grd, 32 * kFansPerBlock, sm, s>>>(fields, rows, tab, exits, p, counters);
    else if (raw)
        k_trace_raster<false, true><<<grd, 32 * kFansPerBlock, sm, s>>>(fields, rows, tab, exits, p, counters);
    else
        k_trace_raster<false, false><<<grd, 32 * kFansPerBlock, sm, s>>>(fields, rows, tab, exits, p, counters);
}

int trace_items(int N, int *nwarps)
{
    const int nw = (N - 2 + 30) / 31;
    if (nwarps) *nwarps = nw;
    return nw * ((N + kFansPerBlock - 1) / kFansPerBlock);
}

template <bool LOSSY, bool RAW>
static int grouped_blocks_of(int max_ny)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_grouped<LOSSY, RAW>, 32 * kFansPerBlock,
                                                      (size_t)max_ny * sizeof(int4)) != cudaSuccess)
        return 0;
    return sms * per_sm;
}

int trace_grouped_blocks(bool lossy, bool raw, int max_ny)
{
    if (lossy && raw) return grouped_blocks_of<true, true>(max_ny);
    if (lossy) return grouped_blocks_of<true, false>(max_ny);
    if (raw) return grouped_blocks_of<false, true>(max_ny);
    return grouped_blocks_of<false, false>(max_ny);
}

void launch_trace_grouped(const TraceGroup &g, int max_ny, int blocks, int *next, bool lossy, bool raw, cudaStream_t s)
{
    const int grd = blocks < g.total ? blocks : g.total;
    const size_t sm = (size_t)max_ny * sizeof(int4);
    if (lossy && raw)
        k_trace_grouped<true, true><<<grd, 32 * kFansPerBlock, sm, s>>>(g, next);
    else if (lossy)
        k_trace_grouped<true, false><<<grd, 32 * kFansPerBlock, sm, s>>>(g, next);
    else if (raw)
        k_trace_grouped<false, true><<<grd, 32 * kFansPerBlock, sm, s>>>(g, next);
    else
        k_trace_grouped<false, false><<<grd, 32 * kFansPerBlock, sm, s>>>(g, next);
}

// rows[iy] = (compact index of the row's first mask node, first ix, last ix); empty rows
// get first ix > last ix. The mask is a disc, so each row's mask nodes are contiguous.
__global__ void k_mask_rows(const int *__restrict__ node2x, int nx, int ny, int4 *__restrict__ rows)
{
    int iy = blockIdx.x * blockDim.x + threadIdx.x;
    if (iy >= ny) return;
    int first = -1, last = -2, off = 0;
    for (int ix = 0; ix < nx; ix++) {
        int k = node2x[iy * nx + ix];
        if (k >= 0) {
            if (first < 0) { first = ix; off = k; }
            last = ix;
        }
    }
    rows[iy] = make_int4(off, first < 0 ? 1 : first, first < 0 ? 0 : last, 0);
}

void launch_mask_rows(const int *node2x, int nx, int ny, int4 *rows, cudaStream_t s)
{
    k_mask_rows<<<(ny + 127) / 128, 128, 0, s>>>(node2x, nx, ny, rows);
}

// ---------------------------------------------------------------- a4

// Angular density of every entry (the back-projection's tensor-core operand synthesis forms
// the same values itself, from the same expression, and does not need this array).
__global__ void k_dgamma(const TabEntry *__restrict__ tab, float *__restrict__ dg, int N, int X)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)N * X) return;
    int e = (int)(i / X), k = (int)(i % X);
    const TabEntry &tp = tab[(size_t)((e + 1) % N) * X + k];
    const TabEntry &tm = tab[(size_t)((e + N - 1) % N) * X + k];
    dg[i] = (tp.idk == kUncovered || tm.idk == kUncovered) ? 0.f : dgamma_of(tp.gam, tm.gam);
}

void launch_dgamma(const TabEntry *tab, float *dg, int N, int X, cudaStream_t s)
{
    size_t n = (size_t)N * X;
    k_dgamma<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tab, dg, N, X);
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

// An angle difference d in (-4 pi, 4 pi) taken to [0, 2 pi) by whole turns.
__device__ __forceinline__ double wrap_turn(double d)
{
    const double TWO_PI = 6.283185307179586476925;
    if (d < 0.0) d += TWO_PI;
    if (d < 0.0) d += TWO_PI;
    if (d >= TWO_PI) d -= TWO_PI;
    if (d >= TWO_PI) d -= TWO_PI;
    return d;
}

// Angle of the receiver m ring places after transducer e (r = (e + m) mod N) relative to it,
// in [0, 2 pi), increasing with m: m steps of step = 2 pi / N on the uniform ring (no FP64
// division or rounding to whole turns: FP64 is slow on this GPU), else the difference of the
// caller's position angles.
__device__ __forceinline__ double recv_rel_m(int m, int e, int N, double step, const double *beta, double be)
{
    return beta ? wrap_turn(beta[(e + m) % N] - be) : (double)m * step;
}

// Position angle of transducer e.
__device__ __forceinline__ double xducer_angle(int e, int N, double step, const double *beta)
{
    return beta ? beta[e] : (double)e * step;
}

// For every receiver r != e of fan e, the first pair of consecutive fan rays (j, j + 1),
// j = 1..N-2, whose exit angles th (relative to beta_e, in [0, 2 pi)) bracket beta_r, as
// first[r] = j, or INT_MAX when no pair does. relt[m] is the receiver angle relative to beta_e
// of ring place m (increasing in m). Each pair marks the receivers between its two exit
// angles (a binary search for the first, then the run up to the larger angle) and the
// smallest j wins, so a fan costs O(N log N) rather than a scan over the pairs per receiver.
// Called by the whole block.
__device__ void first_brackets(const float *th, const float *relt, int N, int e, int *first)
{
    for (int r = threadIdx.x; r < N; r += blockDim.x) first[r] = INT_MAX;
    __syncthreads();
    for (int j = 1 + threadIdx.x; j <= N - 2; j += blockDim.x) {
        const float tj = th[j - 1], tk = th[j];
        if (tj == tk) continue;
        const float lo = fminf(tj, tk), hi = fmaxf(tj, tk);
        int a = 1, b = N;   // first ring place m in [1, N - 1] with relt[m] >= lo (N: none)
        while (a < b) {
            const int c = (a + b) >> 1;
            if (relt[c] < lo) a = c + 1; else b = c;
        }
        for (int m = a; m <= N - 1 && relt[m] <= hi; m++) atomicMin(&first[(e + m) % N], j);
    }
    __syncthreads();
}

__global__ void k_direct_green(const float4 *__restrict__ exits, int N, const double *__restrict__ beta, float fhi,
                               float flo, float C, float2 *__restrict__ g, unsigned long long *counters)
{
    extern __shared__ float4 ex[];
    double *reld = reinterpret_cast<double *>(ex + (N - 1));   // receiver angle relative to beta_e by ring place
    double *thd = reld + N;                                    // exit angle relative to beta_e, in [0, 2 pi)
    float *th = reinterpret_cast<float *>(thd + (N - 1));      // thd rounded to float
    float *relt = th + (N - 1);                                // reld rounded to float
    int *first = reinterpret_cast<int *>(relt + N);            // first bracketing pair per receiver
    const int e = blockIdx.x;
    const double step = 6.283185307179586476925 / N, be = xducer_angle(e, N, step, beta);
    for (int q = threadIdx.x; q < N - 1; q += blockDim.x) {
        float4 v = exits[(size_t)e * (N - 1) + q];
        ex[q] = v;
        thd[q] = wrap_turn((double)v.x - be);
        th[q] = (float)thd[q];
    }
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        reld[m] = recv_rel_m(m, e, N, step, beta, be);
        relt[m] = (float)reld[m];
    }
    __syncthreads();
    first_brackets(th, relt, N, e, first);
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
        if (r == e) { g[(size_t)e * N + r] = make_float2(0.f, 0.f); continue; }
        const double td = reld[(r - e + N) % N];
        const float t = (float)td;
        // first consecutive pair (j, j+1) whose exit angles bracket beta_r
        const int found = first[r] == INT_MAX ? -1 : first[r];
        float T, a;
        int K;
        if (found > 0) {
            float4 A = ex[found - 1], B = ex[found];
            // the bracket fraction from the exit angles in double precision
            const double ta = thd[found - 1], tb = thd[found];
            const double fr = (td - ta) / (tb - ta);
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

void launch_direct_green(const float4 *exits, int N, const double *beta, double f, double c0, float2 *g,
                         unsigned long long *counters, cudaStream_t s)
{
    float fhi = (float)f, flo = (float)(f - (double)fhi);
    float C = (float)(1.0 / sqrt(8.0 * 3.14159265358979323846 * (2.0 * 3.14159265358979323846 * f) / c0));
    size_t smem = (size_t)(N - 1) * (sizeof(float4) + sizeof(double) + sizeof(float)) +
                  (size_t)N * (sizeof(double) + sizeof(float) + sizeof(int));   // <= 180 KB at N = 4095
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_direct_green, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_direct_green<<<N, 512, smem, s>>>(exits, N, beta, fhi, flo, C, g, counters);
}

// ---------------------------------------------------------------- ray linking

// One ray from (x, y) to the ring by one thread: the Heun and paraxial step of k_trace_raster
// (same normalisations, the same compensated sums of the position and T and plain sums of
// the momentum and the paraxial ray, the same reciprocals, the same final partial step)
// without its rasterisation and straight-line shortcuts. The initial direction is formed in double so that a secant
// iteration on it is not limited by FP32 rounding of the angle. Returns false when the ray
// does not reach the ring within p.maxs steps.
template <bool LOSSY, bool RAW>
__device__ bool trace_one(const float *__restrict__ F, const RayParams &p, float x, float y, double gam0,
                          float &theta, float &Tout, float &aout, int &Kout)
{
    const float ds = p.ds, hds = 0.5f * p.ds, R2 = p.R * p.R;
    Fv F1;
    field_eval<LOSSY, RAW>(F, p, x, y, F1);
    double sd, cd;
    sincos(gam0, &sd, &cd);
    float px = F1.n * (float)cd, py = F1.n * (float)sd, dpx = -F1.n * (float)sd, dpy = F1.n * (float)cd;
    float dxx = 0.f, dxy = 0.f, T = 0.f, Tc = 0.f, B = 0.f, Bc = 0.f;
    float cx = 0.f, cy = 0.f;
    float sc1 = 0.f, Jlast = 0.f;
    int K = 0;
    for (int i = 0; i < p.maxs; i++) {
        const float n = F1.n, in = rcp_ap(n);
        const float sc = n * rsqrtf(px * px + py * py);
        px *= sc; py *= sc;
        const float qx = px * in, qy = py * in;
        Fv F2;
        field_eval<LOSSY, RAW>(F, p, x + ds * qx, y + ds * qy, F2);
        const float na = F2.n, ina = rcp_ap(na);
        float pax = px + ds * F1.gx, pay = py + ds * F1.gy;
        const float sca = na * rsqrtf(pax * pax + pay * pay);
        pax *= sca; pay *= sca;
        const float qax = pax * ina, qay = pay * ina;
        const float sx = qx + qax, sy = qy + qay, rs = rsqrtf(sx * sx + sy * sy);
        const float dirx = sx * rs, diry = sy * rs;
        const float ddpx = hds * (F1.gx + F2.gx), ddpy = hds * (F1.gy + F2.gy);
        const float gd = F1.gx * dxx + F1.gy * dxy, pd = px * dpx + py * dpy;
        const float qdxx = in * (dpx - px * gd * in), qdxy = in * (dpy - py * gd * in);
        const float w1 = in * (pd * in - gd);
        const float qdpx = F1.hxx * dxx + F1.hxy * dxy + F1.gx * w1;
        const float qdpy = F1.hxy * dxx + F1.hyy * dxy + F1.gy * w1;
        const float dpax = dpx + ds * qdpx, dpay = dpy + ds * qdpy;
        const float dxax = dxx + ds * qdxx, dxay = dxy + ds * qdxy;
        const float gda = F2.gx * dxax + F2.gy * dxay, pda = pax * dpax + pay * dpay;
        const float qdxax = ina * (dpax - pax * gda * ina), qdxay = ina * (dpay - pay * gda * ina);
        const float w2 = ina * (pda * ina - gda);
        const float qdpax = F2.hxx * dxax + F2.hxy * dxay + F2.gx * w2;
        const float qdpay = F2.hxy * dxax + F2.hyy * dxay + F2.gy * w2;
        const float ddxx = hds * (qdxx + qdxax), ddxy = hds * (qdxy + qdxay);
        const float ddpx2 = hds * (qdpx + qdpax), ddpy2 = hds * (qdpy + qdpay);
        const float xn = x + ds * dirx, yn = y + ds * diry;
        field_eval<LOSSY, RAW>(F, p, xn, yn, F2);
        float inc = hds * (F1.nr + F2.nr), incB = LOSSY ? hds * (F1.al + F2.al) : 0.f;
        const bool last = xn * xn + yn * yn >= R2;
        if (last) {
            // as in k_trace_raster: a first step starts on the ring (|x|^2 - R^2 = 0)
            float b = x * dirx + y * diry, cc = i == 0 ? 0.f : x * x + y * y - R2;
            float disc = b * b - cc;
            float t = -b + sqrtf(disc > 0.f ? disc : 0.f);
            t = fminf(fmaxf(t, 0.f), ds);
            float fr = t / ds;
            x = x + t * dirx; y = y + t * diry;
            inc *= fr;
            incB *= fr;
            dxx += fr * ddxx; dxy += fr * ddxy;
            dpx += fr * ddpx2; dpy += fr * ddpy2;
            px += fr * ddpx; py += fr * ddpy;
            field_eval<LOSSY, RAW>(F, p, x, y, F2);
        } else {
            kadd(x, cx, ds * dirx); kadd(y, cy, ds * diry);
            px += ddpx; py += ddpy;
            dxx += ddxx; dxy += ddxy;
            dpx += ddpx2; dpy += ddpy2;
        }
        kadd(T, Tc, inc);
        if (LOSSY) kadd(B, Bc, incB);
        F1 = F2;
        const float rp = rsqrtf(px * px + py * py), tx = px * rp, ty = py * rp;
        const float J = dxx * ty - dxy * tx;
        if (i == 0) { sc1 = sqrtf(F1.nr * fabsf(J) / ds); Jlast = J; }
        else if (J * Jlast < 0.f) K++;
        if (J != 0.f) Jlast = J;
        if (last) {
            theta = atan2f(y, x);
            Tout = T;
            aout = sc1 * rsqrtf(F1.nr * fabsf(J)) * (LOSSY ? expf(-B) : 1.f);
            Kout = K;
            return true;
        }
    }
    return false;
}

// Linked rays of the direct term (Sec. 4.4, Sec. 6.3.2), in two kernels.
//
// Linking, step 1, one block per transducer: the first bracketing pair of fan rays of every
// receiver (as in k_direct_green), or the nearest fan ray where none brackets it, kept in the
// unused first slot of linked[e][r] as j (> 0) or -j; the diagonal is zeroed.
__global__ void k_link_brackets(const float4 *__restrict__ exits, int N, const double *__restrict__ beta,
                                float4 *__restrict__ linked)
{
    extern __shared__ float4 ex_s[];
    float *th = reinterpret_cast<float *>(ex_s);
    float *relt = th + (N - 1);
    int *first = reinterpret_cast<int *>(relt + N);
    const int e = blockIdx.x;
    const double step = 6.283185307179586476925 / N, be = xducer_angle(e, N, step, beta);
    for (int q = threadIdx.x; q < N - 1; q += blockDim.x)
        th[q] = (float)wrap_turn((double)exits[(size_t)e * (N - 1) + q].x - be);
    for (int m = threadIdx.x; m < N; m += blockDim.x) relt[m] = (float)recv_rel_m(m, e, N, step, beta, be);
    __syncthreads();
    first_brackets(th, relt, N, e, first);
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r != e) {
            int code = first[r];
            if (code == INT_MAX) {
                const float t = relt[(r - e + N) % N];
                int best = 1;
                float bd = 1e30f;
                for (int j = 1; j <= N - 1; j++) {
                    float d = fabsf(th[j - 1] - t);
                    if (d < bd) { bd = d; best = j; }
                }
                code = -best;
            }
            v.x = __int_as_float(code);
        }
        linked[(size_t)e * N + r] = v;
    }
}

// Linking, step 2, one thread per (transducer, receiver) pair; a block's four warps take the
// same 32 receiver offsets m = r - e of four neighbouring transducers, so their rays, rotated
// by one ring step, share L1 lines. From the bracketing fan rays a secant on the initial
// angle, kept inside the bracket (regula falsi with the Illinois weighting), stops when the
// exit lies within tol radians of beta_r (at most maxit new rays); T and a are then
// interpolated in exit angle between the two bracketing rays to beta_r exactly, K taken from
// the nearer; linked[e][r] = (0, T, a, K) serves every frequency of the trace. Unbracketed
// receivers take the nearest fan ray; those and the pairs that stopped on maxit are counted
// in counters[1].
template <bool LOSSY, bool RAW>
__global__ __launch_bounds__(128, 4) void k_link_rays(const float *__restrict__ F, RayParams p,
                                                   const float4 *__restrict__ exits, int maxit, double tol,
                                                   float4 *__restrict__ linked, unsigned long long *counters)
{
    const int N = p.N;
    const int e = blockIdx.y * 4 + (threadIdx.x >> 5), m = blockIdx.x * 32 + (threadIdx.x & 31) + 1;
    if (e >= N || m > N - 1) return;
    const int r = (e + m) % N;
    const double PI = 3.14159265358979323846, TWO_PI = 2.0 * PI;
    const double step = TWO_PI / N, be = xducer_angle(e, N, step, p.beta);
    const double td = recv_rel_m(m, e, N, step, p.beta, be);
    float4 *slot = linked + (size_t)e * N + r;
    const int code = __float_as_int(slot->x);
    const float4 *ex = exits + (size_t)e * (N - 1);
    auto rel = [&](double ang) { return wrap_turn(ang - be); };
    double T, a;
    int K;
    if (code > 0) {
        const int found = code;
        const float xe = (float)(p.R * cos(be)), ye = (float)(p.R * sin(be));
        const float4 A = ex[found - 1], Bq = ex[found];
        // bracketing secant (regula falsi, Illinois weighting): every new ray starts between
        // the two bracketing rays, so it points inward like the fan's
        double ga = be + PI / 2 + PI * found / N, gb = be + PI / 2 + PI * (found + 1) / N;
        double fa = rel(A.x) - td, fb = rel(Bq.x) - td, wa = fa, wb = fb;
        double Ta = A.y, Tb = Bq.y, aa = A.z, ab = Bq.z;
        int Ka = (int)A.w, Kb = (int)Bq.w, it = 0, side = 0;
        while (fabs(fa) > tol && fabs(fb) > tol && it < maxit && wb != wa) {
            const double gc = (ga * wb - gb * wa) / (wb - wa);
            float thc, Tc, ac;
            int Kc;
            if (!trace_one<LOSSY, RAW>(F, p, xe, ye, gc, thc, Tc, ac, Kc)) break;
            double fc = rel(thc) - td;
            if (fc > PI) fc -= TWO_PI;
            if (fc < -PI) fc += TWO_PI;
            it++;
            if ((fc > 0) == (fb > 0)) {
                gb = gc; fb = fc; wb = fc; Tb = Tc; ab = ac; Kb = Kc;
                if (side == -1) wa *= 0.5;
                side = -1;
            } else {
                ga = gc; fa = fc; wa = fc; Ta = Tc; aa = ac; Ka = Kc;
                if (side == 1) wb *= 0.5;
                side = 1;
            }
        }
        if (fabs(fa) > tol && fabs(fb) > tol) atomicAdd(&counters[1], 1ull);
        const double fr = (fb == fa) ? 0.0 : -fa / (fb - fa);
        T = Ta + fr * (Tb - Ta);
        a = aa + fr * (ab - aa);
        K = fabs(fa) <= fabs(fb) ? Ka : Kb;
    } else {
        const float4 A = ex[-code - 1];
        T = A.y; a = A.z; K = (int)A.w;
        atomicAdd(&counters[1], 1ull);
    }
    *slot = make_float4(0.f, (float)T, (float)a, (float)K);
}

// g[e][r] = C a exp(i 2 pi (f T - K/4 + 1/8)) from the linked rays' (-, T, a, K); 0 on the diagonal
__global__ void k_green_linked(const float4 *__restrict__ linked, int N, float fhi, float flo, float C,
                               float2 *__restrict__ g)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)N * N) return;
    const float4 v = linked[i];
    if (i / N == i % N) { g[i] = make_float2(0.f, 0.f); return; }
    float sn, cs;
    sincospif(2.f * phase_cycles(v.y, (int)v.w, fhi, flo), &sn, &cs);
    g[i] = make_float2(C * v.z * cs, C * v.z * sn);
}

void launch_green_linked(const float4 *linked, int N, double f, double c0, float2 *g, cudaStream_t s)
{
    float fhi = (float)f, flo = (float)(f - (double)fhi);
    float C = (float)(1.0 / sqrt(8.0 * 3.14159265358979323846 * (2.0 * 3.14159265358979323846 * f) / c0));
    const size_t n = (size_t)N * N;
    k_green_linked<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(linked, N, fhi, flo, C, g);
}

void launch_link_rays(const float *fields, const RayParams &p, const float4 *exits, int maxit, float4 *linked,
                      unsigned long long *counters, bool lossy, bool raw, cudaStream_t s)
{
    const size_t smem = (size_t)(p.N - 1) * sizeof(float) + (size_t)p.N * (sizeof(float) + sizeof(int));   // <= 49 KB
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_link_brackets, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_link_brackets<<<p.N, 256, smem, s>>>(exits, p.N, p.beta, linked);
    const double tol = 1e-6;
    const dim3 grd((p.N - 1 + 31) / 32, (p.N + 3) / 4);
    if (lossy && raw)
        k_link_rays<true, true><<<grd, 128, 0, s>>>(fields, p, exits, maxit, tol, linked, counters);
    else if (lossy)
        k_link_rays<true, false><<<grd, 128, 0, s>>>(fields, p, exits, maxit, tol, linked, counters);
    else if (raw)
        k_link_rays<false, true><<<grd, 128, 0, s>>>(fields, p, exits, maxit, tol, linked, counters);
    else
        k_link_rays<false, false><<<grd, 128, 0, s>>>(fields, p, exits, maxit, tol, linked, counters);
}

// ---------------------------------------------------------------- table I/O

// counters[0] gains the number of covered entries (a > 0).
__global__ void k_set_tables(const float *T, const float *a, const float *gam, const uint8_t *K, TabEntry *tab,
                             size_t n, unsigned long long *counters)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    bool cov = false;
    if (i < n) {
        TabEntry t;
        float av = a[i];
        cov = av > 0.f;
        t.idk = cov ? (uint32_t)K[i] : kUncovered;
        t.T = T[i];
        t.a = av;
        t.gam = gam[i];
        tab[i] = t;
    }
    const unsigned b = __ballot_sync(0xffffffffu, cov);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&counters[0], (unsigned long long)__popc(b));
}

void launch_set_tables(const float *T, const float *a, const float *gam, const uint8_t *K, TabEntry *tab, size_t n,
                       unsigned long long *counters, cudaStream_t s)
{
    k_set_tables<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(T, a, gam, K, tab, n, counters);
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
