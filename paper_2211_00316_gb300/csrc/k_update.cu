// Steps a7 (residual) and a9 (update), with fixed-order FP64 reductions.
//
// Residual (Eq. residual): R = g_pred - data off the diagonal, R[e,e] = 0, and its
// symmetric part R_s = (R + R^T)/2 that the back-projection consumes.
// Update (Eq. sound_speed_update, Sec. 3.4): dm = -(Delta omega/(2 pi)^3)(m/omega) Re grad,
// grad = 2 (P0 + s P1), m <- m + tau dm on the mask, c = m^-1/2, water outside the mask.
// The minus sign follows the stationarity condition grad F + H dm = 0 with H ~ 2 pi delta.
#include "rbx_internal.cuh"

namespace rbx {

constexpr int RB = 256;

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = RB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_max(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = RB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

int residual_blocks(int N) { return (int)(((size_t)N * N + RB - 1) / RB); }
int update_blocks(int nx, int ny) { return (nx * ny + RB - 1) / RB; }

__device__ __forceinline__ float2 resid_at(const float2 *gdir, const float2 *D, const float2 *data, int N, int e, int r)
{
    if (e == r) return make_float2(0.f, 0.f);
    size_t i = (size_t)e * N + r;
    float2 g = gdir[i], d = D[i], m = data[i];
    return make_float2((g.x + d.x) - m.x, (g.y + d.y) - m.y);
}

// red layout: [0, nb) partial sums of |R|^2; red[nb + 0] = total (written by k_final_sum)
__global__ __launch_bounds__(RB) void k_residual(const float2 *__restrict__ gdir, const float2 *__restrict__ D,
                                                 const float2 *__restrict__ data, int N, float2 *__restrict__ R,
                                                 float2 *__restrict__ Rs, double *__restrict__ red)
{
    __shared__ double sh[RB];
    size_t i = blockIdx.x * (size_t)RB + threadIdx.x;
    double n2 = 0;
    if (i < (size_t)N * N) {
        int e = (int)(i / N), r = (int)(i % N);
        float2 a = resid_at(gdir, D, data, N, e, r), b = resid_at(gdir, D, data, N, r, e);
        if (R) R[i] = a;
        Rs[i] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
        n2 = (double)a.x * a.x + (double)a.y * a.y;
    }
    double s = block_sum(n2, sh);
    if (threadIdx.x == 0) red[blockIdx.x] = s;
}

// Fixed-order sum of the block partials by one block: thread t adds partials t, t + RB, ...
// in turn, then the block tree (the order depends on n only, so results repeat bit for bit).
__global__ __launch_bounds__(RB) void k_final_sum(const double *__restrict__ part, int n, double *__restrict__ out)
{
    __shared__ double sh[RB];
    double v = 0;
    for (int i = threadIdx.x; i < n; i += RB) v += part[i];
    const double s = block_sum(v, sh);
    if (threadIdx.x == 0) *out = s;
}

void launch_residual(const float2 *gdir, const float2 *D, const float2 *data, int N, float2 *R, float2 *Rs,
                     double *red, cudaStream_t s)
{
    int nb = residual_blocks(N);
    k_residual<<<nb, RB, 0, s>>>(gdir, D, data, N, R, Rs, red);
    k_final_sum<<<1, RB, 0, s>>>(red, nb, red + nb);
}

__global__ void k_symmetrize(const float2 *__restrict__ R, int N, float2 *__restrict__ Rs)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)N * N) return;
    int e = (int)(i / N), r = (int)(i % N);
    float2 a = R[i], b = R[(size_t)r * N + e];
    Rs[i] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
}

void launch_symmetrize(const float2 *R, int N, float2 *Rs, cudaStream_t s)
{
    size_t n = (size_t)N * N;
    k_symmetrize<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(R, N, Rs);
}

// out[x] = scale * (g0 + s g1) (mode 0, s = -1 or +1 by weight_mode, scale = 2)
//        = scale * g0          (mode 1, scale = omega^2 dA)
__global__ void k_combine(const float2 *__restrict__ gpart, int X, int mode, float sgn, double scale,
                          float2 *__restrict__ out)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= X) return;
    float2 g0 = gpart[x];
    double re = g0.x, im = g0.y;
    if (mode == 0) {
        float2 g1 = gpart[(size_t)X + x];
        re += sgn * (double)g1.x;
        im += sgn * (double)g1.y;
    }
    out[x] = make_float2((float)(scale * re), (float)(scale * im));
}

void launch_combine_adjoint(const float2 *gpart, int X, int mode, int weight_mode, double scale, float2 *out,
                            cudaStream_t s)
{
    k_combine<<<(X + 255) / 256, 256, 0, s>>>(gpart, X, mode, weight_mode == 0 ? -1.f : 1.f, scale, out);
}

// plain adjoint on a lossy medium: out[x] = dA conj(Upsilon_m) g0[x], Upsilon_m = omega c k~
__global__ void k_combine_lossy(const float2 *__restrict__ gpart, const float *__restrict__ c,
                                const float *__restrict__ alpha0, const int *__restrict__ idx, int X, double w,
                                double wy, double tn, double dA, float2 *__restrict__ out)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= X) return;
    const int k = idx[x];
    const double cc = c[k], al = wy * (double)alpha0[k];
    const double ur = w * w + w * cc * al * tn, ui = -w * cc * al;       // conj(Upsilon_m)
    const double gr = gpart[x].x, gi = gpart[x].y;
    out[x] = make_float2((float)(dA * (ur * gr - ui * gi)), (float)(dA * (ur * gi + ui * gr)));
}

void launch_combine_adjoint_lossy(const float2 *gpart, const float *c, const int *idx, int X, double f, double dA,
                                  const Lossy &ab, float2 *out, cudaStream_t s)
{
    const double PI = 3.14159265358979323846, w = 2 * PI * f;
    k_combine_lossy<<<(X + 255) / 256, 256, 0, s>>>(gpart, c, ab.alpha0, idx, X, w, pow(w, ab.y),
                                                    tan(PI * ab.y / 2), dA, out);
}

// red layout (nb = update blocks): [0,nb) sum dc^2, [nb,2nb) max |dc|, [2nb,3nb) sum dm^2,
// totals at [3nb], [3nb+1], [3nb+2]
// Lossless: dm = -(Delta omega/(2 pi)^3) (m/omega) Re grad. Lossy (alpha0 != nullptr): the node
// factor m/omega becomes k (1/c + y tan(pi y/2) omega^(y-1) alpha0) / Upsilon_m with
// k = omega/c + alpha0 tan(pi y/2) omega^y (the derivative of |kbar| in Sec. 3.3 and
// Eq. scattering-potential), complex, and dm = -(Delta omega/(2 pi)^3) Re{factor grad}.
__global__ __launch_bounds__(RB) void k_update(const float2 *__restrict__ gpart, const int *__restrict__ node2x, int X,
                                               int nxy, float sgn, double pref_over_w, double tau, float c0,
                                               float *__restrict__ c, double *__restrict__ red,
                                               unsigned long long *counters, const float *__restrict__ alpha0,
                                               double w, double y, double wy, double tn, double *__restrict__ acc,
                                               int mode)
{
    __shared__ double sh[RB];
    int k = blockIdx.x * RB + threadIdx.x;
    double dc2 = 0, dcm = 0, dm2 = 0;
    if (k < nxy) {
        int xi = node2x[k];
        if (xi < 0) {
            c[k] = c0;
        } else {
            double grad = 2.0 * ((double)gpart[xi].x + sgn * (double)gpart[(size_t)X + xi].x);
            double cold = c[k];
            double m = 1.0 / (cold * cold);
            double dm;
            if (alpha0) {
                const double a0 = alpha0[k], al = a0 * wy;
                const double gim = 2.0 * ((double)gpart[xi].y + sgn * (double)gpart[(size_t)X + xi].y);
                const double kr = w / cold + al * tn;
                const double num = kr * (1.0 / cold + y * tn * (wy / w) * a0);
                const double ur = w * w + w * cold * al * tn, ui = w * cold * al, un = ur * ur + ui * ui;
                const double fr = num * ur / un, fi = -num * ui / un;
                dm = -pref_over_w * w * (fr * grad - fi * gim);
            } else {
                dm = -pref_over_w * m * grad;
            }
            // frequency sets: mode 1 starts the sum of the set's search directions, mode 2 adds
            // to it (the model is not touched), mode 3 adds the last one and applies the step;
            // mode 0 is a single frequency
            if (mode == 1 || mode == 2) {
                acc[xi] = (mode == 1 ? 0.0 : acc[xi]) + dm;
            } else {
                if (mode == 3) dm += acc[xi];
                double mn = m + tau * dm;
                if (!(mn > 0.0) || !isfinite(mn)) {
                    atomicAdd(&counters[4], 1ull);
                    mn = m;
                }
                float cn = (float)(1.0 / sqrt(mn));
                c[k] = cn;
                double dc = (double)cn - cold;
                dc2 = dc * dc;
                dcm = fabs(dc);
                dm2 = dm * dm;
            }
        }
    }
    double s1 = block_sum(dc2, sh), s2 = block_max(dcm, sh), s3 = block_sum(dm2, sh);
    if (threadIdx.x == 0) {
        red[blockIdx.x] = s1;
        red[gridDim.x + blockIdx.x] = s2;
        red[2 * gridDim.x + blockIdx.x] = s3;
    }
}

// The update's three block partials (sum dc^2, max |dc|, sum dm^2) in the fixed order of
// k_final_sum.
__global__ __launch_bounds__(RB) void k_final_update(const double *__restrict__ red, int nb, double *__restrict__ out)
{
    __shared__ double sh[RB];
    double s1 = 0, s2 = 0, s3 = 0;
    for (int i = threadIdx.x; i < nb; i += RB) {
        s1 += red[i];
        s2 = fmax(s2, red[nb + i]);
        s3 += red[2 * nb + i];
    }
    s1 = block_sum(s1, sh);
    s2 = block_max(s2, sh);
    s3 = block_sum(s3, sh);
    if (threadIdx.x == 0) {
        out[0] = s1;
        out[1] = s2;
        out[2] = s3;
    }
}

void launch_update(const float2 *gpart, const int *node2x, int nx, int ny, int X, int weight_mode, double f,
                   double df, double tau, double c0, float *c, double *red, unsigned long long *counters,
                   const Lossy &ab, double *acc, int mode, cudaStream_t s)
{
    const double PI = 3.14159265358979323846;
    double w = 2 * PI * f, dw = 2 * PI * df;
    double pref = dw / (8 * PI * PI * PI);
    int nb = update_blocks(nx, ny);
    const double wy = ab.alpha0 ? pow(w, ab.y) : 0.0, tn = ab.alpha0 ? tan(PI * ab.y / 2) : 0.0;
    k_update<<<nb, RB, 0, s>>>(gpart, node2x, X, nx * ny, weight_mode == 0 ? -1.f : 1.f, pref / w, tau, (float)c0, c,
                               red, counters, ab.alpha0, w, ab.y, wy, tn, acc, mode);
    k_final_update<<<1, RB, 0, s>>>(red, nb, red + 3 * nb);
}

}  // namespace rbx

namespace rbx {

// out = a + b off the diagonal, 0 on it (predicted data g_dir + D).
__global__ void k_add_offdiag(const float2 *__restrict__ a, const float2 *__restrict__ b, int N, float2 *__restrict__ out)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)N * N) return;
    int e = (int)(i / N), r = (int)(i % N);
    out[i] = e == r ? make_float2(0.f, 0.f) : make_float2(a[i].x + b[i].x, a[i].y + b[i].y);
}

void launch_add_offdiag(const float2 *a, const float2 *b, int N, float2 *out, cudaStream_t s)
{
    size_t n = (size_t)N * N;
    k_add_offdiag<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, b, N, out);
}

}  // namespace rbx

namespace rbx {

// slot = (|R|^2, sum dc^2, max |dc|, sum dm^2, uncovered, clamped, bad rays, CAS bound,
//         non-positive m, bad model, tensor-core timeout, 0)
__global__ void k_snapshot(const double *r2, const double *upd3, const unsigned long long *counters,
                           const unsigned *tc_err, unsigned long long n_entries, double *slot)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    slot[0] = *r2;
    slot[1] = upd3[0];
    slot[2] = upd3[1];
    slot[3] = upd3[2];
    slot[4] = (double)(n_entries - counters[0]);   // counters[0] holds the covered entries
    for (int k = 1; k < 6; k++) slot[4 + k] = (double)counters[k];
    slot[10] = tc_err ? (double)*tc_err : 0.0;
    slot[11] = 0.0;
}

void launch_snapshot(const double *r2, const double *upd3, const unsigned long long *counters, const unsigned *tc_err,
                     unsigned long long n_entries, double *slot, cudaStream_t s)
{
    k_snapshot<<<1, 32, 0, s>>>(r2, upd3, counters, tc_err, n_entries, slot);
}

// dst = (first ? 0 : dst) + src: the residual norm summed over a frequency set
__global__ void k_acc_scalar(const double *__restrict__ src, double *__restrict__ dst, int first)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) dst[0] = (first ? 0.0 : dst[0]) + src[0];
}

void launch_acc_scalar(const double *src, double *dst, bool first, cudaStream_t s)
{
    k_acc_scalar<<<1, 32, 0, s>>>(src, dst, first ? 1 : 0);
}

}  // namespace rbx
