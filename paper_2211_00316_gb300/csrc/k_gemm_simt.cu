// Steps a6-a8 on CUDA cores (FP32): Green's function synthesis and the two complex
// contractions of the update.
//
//  forward (Eqs. perturb1, derivative):  D[e,r] = sum_x G_e[x] G_r[x] v[x]
//  back-projection (Eq. sound_speed_update2), exact two-term factorisation:
//     W_er = 2 (1 + s cos(gamma_e - gamma_r)) = 2 + s (kappa_e conj(kappa_r) + conj(kappa_e) kappa_r),
//     kappa = e^{i gamma}, s = -1 (printed scattering angle) or +1 (isochron); since W and
//     u_e u_r are symmetric in (e, r) the residual may be replaced by R_s = (R + R^T)/2, so
//     grad[x] = 2 sum_e u_e P0[x,e] + 2 s sum_e kappa_e u_e P1[x,e],
//     P0 = U^T R_s, P1 = (conj(kappa) U)^T R_s,
//  i.e. a complex GEMM with the two stacks as rows and a fused row-dot epilogue.
//
// Tiles: 64 x 64 complex outputs per 256-thread block, 4 x 4 complex per thread, K chunks
// of 16. The forward is complex-symmetric: only tiles with e-tile <= r-tile are computed,
// split over the mask nodes; a fixed-order reduction mirrors them (D exactly symmetric).
#include "rbx_internal.cuh"

namespace rbx {

__device__ __forceinline__ float phase_cycles_(float T, int K, float fhi, float flo)
{
    float p = fhi * T;
    float err = fmaf(fhi, T, -p) + flo * T;
    float r = (p - rintf(p)) + err;
    return r + 0.125f - 0.25f * (float)K;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ void cmac(float2 &acc, float2 a, float2 b)
{
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// G_e[x] = (8 pi omega/c0)^(-1/2) a exp(i 2 pi (f T - K/4 + 1/8))      (Eq. 2D_greens)
__global__ void k_synth_fwd(const TabEntry *__restrict__ tab, size_t n, float fhi, float flo, float C,
                            float2 *__restrict__ G)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    TabEntry t = tab[i];
    if (t.idk == kUncovered) { G[i] = make_float2(0.f, 0.f); return; }
    float s, c;
    sincospif(2.f * phase_cycles_(t.T, (int)(t.idk & 0xffu), fhi, flo), &s, &c);
    float A = C * t.a;
    G[i] = make_float2(A * c, A * s);
}

// u_e[x] = dgamma_e[x] / ((8 pi omega/c0)^(-1/2) a) exp(-i 2 pi (f T - K/4 + 1/8))   (Eq. greens-time-reversed)
// kap_e[x] = (cos gamma, sin gamma)
__global__ void k_synth_bp(const TabEntry *__restrict__ tab, const float *__restrict__ dg, size_t n, float fhi,
                           float flo, float C, float2 *__restrict__ U, float2 *__restrict__ kap)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    TabEntry t = tab[i];
    if (t.idk == kUncovered) { U[i] = make_float2(0.f, 0.f); kap[i] = make_float2(1.f, 0.f); return; }
    float s, c;
    sincospif(2.f * phase_cycles_(t.T, (int)(t.idk & 0xffu), fhi, flo), &s, &c);
    float A = dg[i] / (C * t.a);
    U[i] = make_float2(A * c, -A * s);
    float sg, cg;
    sincosf(t.gam, &sg, &cg);
    kap[i] = make_float2(cg, sg);
}

static void fsplit(double f, float &fhi, float &flo)
{
    fhi = (float)f;
    flo = (float)(f - (double)fhi);
}

static float green_const(double f, double c0)
{
    return (float)(1.0 / sqrt(8.0 * 3.14159265358979323846 * (2.0 * 3.14159265358979323846 * f) / c0));
}

void launch_synth_fwd(const TabEntry *tab, int N, int X, double f, double c0, float2 *G, cudaStream_t s)
{
    size_t n = (size_t)N * X;
    float fhi, flo;
    fsplit(f, fhi, flo);
    k_synth_fwd<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tab, n, fhi, flo, green_const(f, c0), G);
}

void launch_synth_bp(const TabEntry *tab, const float *dg, int N, int X, double f, double c0, float2 *U, float2 *kap,
                     cudaStream_t s)
{
    size_t n = (size_t)N * X;
    float fhi, flo;
    fsplit(f, fhi, flo);
    k_synth_bp<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tab, dg, n, fhi, flo, green_const(f, c0), U, kap);
}

// Scattering potential Upsilon_m = omega c k~ (Eq. scattering-potential), with
// k~ = omega/c + alpha0 omega^y (tan(pi y/2) + i) (Eq. szabo_dispersion_equation):
// (omega^2 + omega c alpha tan(pi y/2), omega c alpha), alpha = alpha0 omega^y; omega^2 lossless.
__device__ __forceinline__ double2 upsilon_m(double w, double c, double alpha, double tn)
{
    return make_double2(w * w + w * c * alpha * tn, w * c * alpha);
}

// v[x] = Upsilon_m dA (m - m_s) on the mask: Born weight of the rough part of the model.
__global__ void k_born_rough(const float *__restrict__ c, const double *__restrict__ ns, const int *__restrict__ idx,
                             int X, double w, double dA, const float *__restrict__ alpha0, double wy, double tn,
                             float2 *__restrict__ v)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= X) return;
    int k = idx[q];
    double cc = c[k], n = ns[k];
    double2 u = upsilon_m(w, cc, alpha0 ? wy * (double)alpha0[k] : 0.0, tn);
    double d = dA * (1.0 / (cc * cc) - n * n);
    v[q] = make_float2((float)(u.x * d), (float)(u.y * d));
}

__global__ void k_born_dm(const float *__restrict__ dm, const float *__restrict__ c, const int *__restrict__ idx, int X,
                          double w, double dA, const float *__restrict__ alpha0, double wy, double tn,
                          float2 *__restrict__ v)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= X) return;
    int k = idx[q];
    double2 u = alpha0 ? upsilon_m(w, (double)c[k], wy * (double)alpha0[k], tn) : make_double2(w * w, 0.0);
    double d = dA * (double)dm[k];
    v[q] = make_float2((float)(u.x * d), (float)(u.y * d));
}

static void lossy_factors(const Lossy &ab, double w, double &wy, double &tn)
{
    wy = tn = 0.0;
    if (ab.alpha0) {
        wy = pow(w, ab.y);
        tn = tan(3.14159265358979323846 * ab.y / 2.0);
    }
}

void launch_born_weights_rough(const float *c, const double *ns64, const int *idx, int X, double f, double dA,
                               const Lossy &ab, float2 *v, cudaStream_t s)
{
    double w = 2.0 * 3.14159265358979323846 * f, wy, tn;
    lossy_factors(ab, w, wy, tn);
    k_born_rough<<<(X + 255) / 256, 256, 0, s>>>(c, ns64, idx, X, w, dA, ab.alpha0, wy, tn, v);
}

void launch_born_weights_dm(const float *dm, const float *c, const int *idx, int X, double f, double dA,
                            const Lossy &ab, float2 *v, cudaStream_t s)
{
    double w = 2.0 * 3.14159265358979323846 * f, wy, tn;
    lossy_factors(ab, w, wy, tn);
    k_born_dm<<<(X + 255) / 256, 256, 0, s>>>(dm, c, idx, X, w, dA, ab.alpha0, wy, tn, v);
}

// ---------------------------------------------------------------- forward

constexpr int TM = 64, TK = 16;

int forward_splits(int N, int X)
{
    int T = (N + TM - 1) / TM, pairs = T * (T + 1) / 2;
    int s = (2048 + pairs - 1) / pairs;
    int smax = (X + 255) / 256;
    if (s > smax) s = smax;
    if (s > 64) s = 64;
    return s < 1 ? 1 : s;
}

__global__ __launch_bounds__(256) void k_forward_simt(const float2 *__restrict__ G, const float2 *__restrict__ v, int N,
                                                      int X, int xchunk, float2 *__restrict__ part)
{
    // upper-triangular tile pair from the linear block index
    int T = (N + TM - 1) / TM;
    int b = blockIdx.x, te = 0;
    while (b >= T - te) { b -= T - te; te++; }
    int tr = te + b;
    int split = blockIdx.y;
    int xb = split * xchunk, xe = min(X, xb + xchunk);
    __shared__ float2 As[TK][TM + 1], Bs[TK][TM + 1];
    int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = make_float2(0.f, 0.f);
    int lk = threadIdx.x & 15, lr = threadIdx.x >> 4;
    for (int x0 = xb; x0 < xe; x0 += TK) {
        int x = x0 + lk;
        bool ok = x < xe;
        const float2 vv = ok ? v[x] : make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int row = lr + 16 * q;
            int e = te * TM + row, r = tr * TM + row;
            As[lk][row] = (ok && e < N) ? G[(size_t)e * X + x] : make_float2(0.f, 0.f);
            float2 g = (ok && r < N) ? G[(size_t)r * X + x] : make_float2(0.f, 0.f);
            Bs[lk][row] = make_float2(g.x * vv.x - g.y * vv.y, g.x * vv.y + g.y * vv.x);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; k++) {
            float2 a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) bb[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) cmac(acc[i][j], a[i], bb[j]);
        }
        __syncthreads();
    }
    float2 *P = part + (size_t)split * N * N;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int e = te * TM + ty + 16 * i, r = tr * TM + tx + 16 * j;
            if (e < N && r < N) P[(size_t)e * N + r] = acc[i][j];
        }
}

void launch_forward_simt(const float2 *G, const float2 *v, int N, int X, int splits, float2 *part, cudaStream_t s)
{
    int T = (N + TM - 1) / TM, pairs = T * (T + 1) / 2;
    int xchunk = (X + splits - 1) / splits;
    xchunk = (xchunk + TK - 1) / TK * TK;
    k_forward_simt<<<dim3(pairs, splits), 256, 0, s>>>(G, v, N, X, xchunk, part);
}

// D[e,r] = D[r,e] = sum over splits (fixed order) of the upper-triangle partials.
__global__ void k_forward_reduce(const float2 *__restrict__ part, int N, int splits, float2 *__restrict__ D)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)N * N) return;
    int e = (int)(i / N), r = (int)(i % N);
    if (e > r) return;
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < splits; q++) {
        float2 p = part[(size_t)q * N * N + i];
        acc.x += p.x;
        acc.y += p.y;
    }
    D[(size_t)e * N + r] = acc;
    D[(size_t)r * N + e] = acc;
}

void launch_forward_reduce(const float2 *part, int N, int splits, float2 *D, cudaStream_t s)
{
    size_t n = (size_t)N * N;
    k_forward_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, N, splits, D);
}

// ---------------------------------------------------------------- back-projection

// mode 0 (preconditioned): stack 0 A = U, W = U; stack 1 A = conj(kap) U, W = kap U.
// mode 1 (plain adjoint):  A = W = conj(G) (one stack).
// gpart[stack][x] = sum_e W[e][x] sum_r A[r][x] Rs[r][e], complex.
__global__ __launch_bounds__(256) void k_backproject_simt(const float2 *__restrict__ A, const float2 *__restrict__ kap,
                                                          const float2 *__restrict__ Rs, int N, int X, int mode,
                                                          float2 *__restrict__ gpart)
{
    const int stack = blockIdx.y;
    const int xt = blockIdx.x;
    __shared__ __align__(16) float2 smem[TM * (TM + 1)];   // K tiles, then W tile, then reduction
    float2(*As)[TM + 1] = reinterpret_cast<float2(*)[TM + 1]>(smem);
    float2(*Bs)[TM + 1] = reinterpret_cast<float2(*)[TM + 1]>(smem + TK * (TM + 1));
    float2(*Ws)[TM + 1] = reinterpret_cast<float2(*)[TM + 1]>(smem);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int lx = threadIdx.x & 63, lk = threadIdx.x >> 6;   // loader: 64 columns x 4 rows
    float2 gsum[4];
#pragma unroll
    for (int i = 0; i < 4; i++) gsum[i] = make_float2(0.f, 0.f);
    const int ET = (N + TM - 1) / TM;
    for (int et = 0; et < ET; et++) {
        float2 acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] = make_float2(0.f, 0.f);
        for (int r0 = 0; r0 < N; r0 += TK) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                int k = lk + 4 * q, r = r0 + k;
                int x = xt * TM + lx;
                float2 a = make_float2(0.f, 0.f);
                if (r < N && x < X) {
                    size_t off = (size_t)r * X + x;
                    a = A[off];
                    if (mode == 1) a = conjf2(a);
                    else if (stack == 1) a = cmul(conjf2(kap[off]), a);
                }
                As[k][lx] = a;
                int ec = et * TM + lx;
                Bs[k][lx] = (r < N && ec < N) ? Rs[(size_t)r * N + ec] : make_float2(0.f, 0.f);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < TK; k++) {
                float2 a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; i++) a[i] = As[k][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; j++) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) cmac(acc[i][j], a[i], b[j]);
            }
            __syncthreads();
        }
        // W tile [e][x] through shared memory (coalesced along x)
        for (int q = threadIdx.x; q < TM * TM; q += blockDim.x) {
            int el = q / TM, xl = q % TM;
            int e = et * TM + el, x = xt * TM + xl;
            float2 w = make_float2(0.f, 0.f);
            if (e < N && x < X) {
                size_t off = (size_t)e * X + x;
                w = A[off];
                if (mode == 1) w = conjf2(w);
                else if (stack == 1) w = cmul(kap[off], w);
            }
            Ws[el][xl] = w;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) cmac(gsum[i], Ws[tx + 16 * j][ty + 16 * i], acc[i][j]);
        __syncthreads();
    }
    // fixed-order reduction over the 16 threads that share each x
    float2(*red)[TM + 1] = reinterpret_cast<float2(*)[TM + 1]>(smem);
#pragma unroll
    for (int i = 0; i < 4; i++) red[tx][ty + 16 * i] = gsum[i];
    __syncthreads();
    if (threadIdx.x < TM) {
        int x = xt * TM + threadIdx.x;
        float2 s = make_float2(0.f, 0.f);
        for (int q = 0; q < 16; q++) {
            s.x += red[q][threadIdx.x].x;
            s.y += red[q][threadIdx.x].y;
        }
        if (x < X) gpart[(size_t)stack * X + x] = s;
    }
}

void launch_backproject_simt(const float2 *A, const float2 *kap, const float2 *Rs, int N, int X, int mode,
                             float2 *gpart, cudaStream_t s)
{
    dim3 grd((X + TM - 1) / TM, mode == 0 ? 2 : 1);
    k_backproject_simt<<<grd, 256, 0, s>>>(A, kap, Rs, N, X, mode, gpart);
}

}  // namespace rbx
