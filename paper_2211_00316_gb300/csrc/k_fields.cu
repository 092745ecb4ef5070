// Step a1: mask map, smoothing of the slowness and its derivative fields.
//
// The paper traces rays on a wavenumber map smoothed by an odd moving-average window
// whose width falls from low to high frequency (Sec. 6.2, Sec. 6.3.2) and interpolates
// k, grad k and the Hessian of k onto the rays (Sec. 4.4). With k = omega n the ray path
// does not depend on omega, so the fields are those of the slowness n = 1/c.
//
// These kernels touch the grid a few times (512^2 nodes at the largest workload) and are
// computed in FP64: second differences of a slowness that varies by a few percent lose
// most of their digits in FP32. The results are stored as FP32, 8 floats per node, so a
// bilinear gather of one node reads two aligned float4.
#include "rbx_internal.cuh"

namespace rbx {

// Row-major ordering of mask nodes needs a prefix count; the grid is at most a few
// hundred thousand nodes, so a single block does it in two passes over rows.
__global__ void k_mask_single(int nx, int ny, double dx, double x0, double y0, double r2, int *node2x, int *count)
{
    extern __shared__ int rowcnt[];
    // positions and radii rounded exactly as written (no FMA contraction), so the mask
    // is the same node set as any IEEE double evaluation of |x|^2 <= r^2
    for (int iy = threadIdx.x; iy < ny; iy += blockDim.x) {
        double y = __dadd_rn(y0, __dmul_rn((double)iy, dx));
        int cnt = 0;
        for (int ix = 0; ix < nx; ix++) {
            double x = __dadd_rn(x0, __dmul_rn((double)ix, dx));
            cnt += (__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)) <= r2);
        }
        rowcnt[iy] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int iy = 0; iy < ny; iy++) {
            int c = rowcnt[iy];
            rowcnt[iy] = acc;
            acc += c;
        }
        *count = acc;
    }
    __syncthreads();
    for (int iy = threadIdx.x; iy < ny; iy += blockDim.x) {
        double y = __dadd_rn(y0, __dmul_rn((double)iy, dx));
        int k = rowcnt[iy];
        for (int ix = 0; ix < nx; ix++) {
            double x = __dadd_rn(x0, __dmul_rn((double)ix, dx));
            node2x[iy * nx + ix] = (__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)) <= r2) ? k++ : -1;
        }
    }
}

void launch_mask(const rbx_geometry &g, int *node2x, int *count, cudaStream_t s)
{
    k_mask_single<<<1, 256, g.ny * sizeof(int), s>>>(g.nx, g.ny, g.dx, g.x0, g.y0, g.mask_radius * g.mask_radius,
                                                     node2x, count);
}

__global__ void k_mask_idx(const int *node2x, int nxy, int *idx)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nxy && node2x[k] >= 0) idx[node2x[k]] = k;
}

void launch_mask_idx(const int *node2x, int nxy, int *idx, cudaStream_t s)
{
    k_mask_idx<<<(nxy + 255) / 256, 256, 0, s>>>(node2x, nxy, idx);
}

__device__ __forceinline__ int clampi(int i, int lo, int hi) { return i < lo ? lo : (i > hi ? hi : i); }

// Moving average of width w along x of the slowness 1/c (edges replicated).
__global__ void k_smooth_x(const float *__restrict__ c, double *__restrict__ t, int nx, int ny, int w)
{
    int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y;
    if (ix >= nx) return;
    int h = (w - 1) / 2;
    double s = 0;
    for (int d = -h; d <= h; d++) s += 1.0 / (double)c[iy * nx + clampi(ix + d, 0, nx - 1)];
    t[iy * nx + ix] = s / w;
}

// The same average with the block's row segment and its halo inverted once into shared
// memory (FP64 division is slow on this part: one per node instead of w), summed in the same
// order, so the result is the same bit for bit.
__global__ void k_smooth_x_inv(const float *__restrict__ c, double *__restrict__ t, int nx, int ny, int w)
{
    extern __shared__ double rinv[];   // [blockDim.x + w - 1]
    const int h = (w - 1) / 2, ix0 = blockIdx.x * blockDim.x, iy = blockIdx.y;
    for (int q = threadIdx.x; q < (int)blockDim.x + 2 * h; q += blockDim.x)
        rinv[q] = 1.0 / (double)c[iy * nx + clampi(ix0 - h + q, 0, nx - 1)];
    __syncthreads();
    const int ix = ix0 + threadIdx.x;
    if (ix >= nx) return;
    double s = 0;
    for (int d = -h; d <= h; d++) s += rinv[threadIdx.x + h + d];
    t[iy * nx + ix] = s / w;
}

// Moving average along y (edges replicated).
__global__ void k_smooth_y(const double *__restrict__ t, double *__restrict__ ns64, float *__restrict__ ns, int nx,
                           int ny, int w)
{
    int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y;
    if (ix >= nx) return;
    int h = (w - 1) / 2;
    double s = 0;
    for (int d = -h; d <= h; d++) s += t[clampi(iy + d, 0, ny - 1) * nx + ix];
    s /= w;
    ns64[iy * nx + ix] = s;
    ns[iy * nx + ix] = (float)s;
}

// Moving average of width w along x of an arbitrary map (edges replicated).
__global__ void k_smooth_x_map(const float *__restrict__ a, double *__restrict__ t, int nx, int ny, int w)
{
    int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y;
    if (ix >= nx) return;
    int h = (w - 1) / 2;
    double s = 0;
    for (int d = -h; d <= h; d++) s += (double)a[iy * nx + clampi(ix + d, 0, nx - 1)];
    t[iy * nx + ix] = s / w;
}

__global__ void k_smooth_y_map(const double *__restrict__ t, double *__restrict__ out, int nx, int ny, int w)
{
    int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y;
    if (ix >= nx) return;
    int h = (w - 1) / 2;
    double s = 0;
    for (int d = -h; d <= h; d++) s += t[clampi(iy + d, 0, ny - 1) * nx + ix];
    out[iy * nx + ix] = s / w;
}

// Central differences of the smoothed ray slowness (edge indices clamped). Lossless: the
// smoothed 1/c. Lossy (as != nullptr): n_e = smoothed 1/c + tn * smoothed alpha0 with
// tn = tan(pi y/2) omega^(y-1) (the box filter is linear, so this is the smoothed real
// wavenumber map over omega), and the record's slot 6 holds alpha = wy * smoothed alpha0.
// Integration on the non-smoothed map (c_raw != nullptr): slot 7 holds the non-smoothed
// slowness 1/c (+ tn alpha0 when lossy) and slot 6 the non-smoothed alpha.
__global__ void k_fields(const double *__restrict__ ns, const double *__restrict__ as, double tn, double wy,
                         const float *__restrict__ c_raw, const float *__restrict__ a_raw, float *__restrict__ F,
                         int nx, int ny, double dx)
{
    int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y;
    if (ix >= nx) return;
    auto at = [&](int i, int j) {
        const size_t k = (size_t)clampi(j, 0, ny - 1) * nx + clampi(i, 0, nx - 1);
        return as ? ns[k] + tn * as[k] : ns[k];
    };
    double c = at(ix, iy);
    double fx = (at(ix + 1, iy) - at(ix - 1, iy)) / (2 * dx);
    double fy = (at(ix, iy + 1) - at(ix, iy - 1)) / (2 * dx);
    double fxx = (at(ix + 1, iy) - 2 * c + at(ix - 1, iy)) / (dx * dx);
    double fxy = (at(ix + 1, iy + 1) - at(ix - 1, iy + 1) - at(ix + 1, iy - 1) + at(ix - 1, iy - 1)) / (4 * dx * dx);
    double fyy = (at(ix, iy + 1) - 2 * c + at(ix, iy - 1)) / (dx * dx);
    const size_t k0 = (size_t)iy * nx + ix;
    float al = as ? (float)(wy * as[k0]) : 0.f, nr = 0.f;
    if (c_raw) {
        const double a0 = a_raw ? (double)a_raw[k0] : 0.0;
        nr = (float)(1.0 / (double)c_raw[k0] + tn * a0);
        if (as) al = (float)(wy * a0);
    }
    const size_t nxy = (size_t)nx * ny;
    float4 *o4 = reinterpret_cast<float4 *>(F);
    float2 *o2 = reinterpret_cast<float2 *>(o4 + nxy);
    o4[k0] = make_float4((float)c, (float)fx, (float)fy, (float)fxx);
    o2[k0] = make_float2((float)fxy, (float)fyy);
    o2[nxy + k0] = make_float2(al, nr);
}

void launch_smooth_fields(const rbx_geometry &g, const float *c, int w, double *tmp64, double *ns64, float *ns,
                          float *fields, const Lossy &ab, double f, bool raw, cudaStream_t s)
{
    dim3 blk(128), grd((g.nx + 127) / 128, g.ny);
    const size_t inv_smem = (size_t)(128 + w - 1) * sizeof(double);
    if (inv_smem <= 32768)
        k_smooth_x_inv<<<grd, blk, inv_smem, s>>>(c, tmp64, g.nx, g.ny, w);
    else   // a window over 4000 nodes: invert in the sum
        k_smooth_x<<<grd, blk, 0, s>>>(c, tmp64, g.nx, g.ny, w);
    k_smooth_y<<<grd, blk, 0, s>>>(tmp64, ns64, ns, g.nx, g.ny, w);
    double tn = 0.0, wy = 0.0;
    if (ab.alpha0) {
        const double PI = 3.14159265358979323846, om = 2.0 * PI * f;
        tn = tan(PI * ab.y / 2.0) * pow(om, ab.y - 1.0);
        wy = pow(om, ab.y);
        k_smooth_x_map<<<grd, blk, 0, s>>>(ab.alpha0, tmp64, g.nx, g.ny, w);
        k_smooth_y_map<<<grd, blk, 0, s>>>(tmp64, ab.as64, g.nx, g.ny, w);
    }
    k_fields<<<grd, blk, 0, s>>>(ns64, ab.alpha0 ? ab.as64 : nullptr, tn, wy, raw ? c : nullptr, ab.alpha0, fields, g.nx,
                                 g.ny, g.dx);
}

__global__ void k_check_model(const float *c, int n, unsigned long long *flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        float v = c[i];
        if (!(v > 0.f) || !isfinite(v)) atomicAdd(flag, 1ull);
    }
}

void launch_check_model(const float *c, int n, unsigned long long *flag, cudaStream_t s)
{
    k_check_model<<<(n + 255) / 256, 256, 0, s>>>(c, n, flag);
}

__global__ void k_check_alpha(const float *a, int n, unsigned long long *flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(a[i] >= 0.f && isfinite(a[i]))) atomicAdd(flag, 1ull);
}

void launch_check_alpha(const float *a, int n, unsigned long long *flag, cudaStream_t s)
{
    k_check_alpha<<<(n + 255) / 256, 256, 0, s>>>(a, n, flag);
}

__global__ void k_fill(float *p, float v, size_t n)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

void launch_fill(float *p, float v, size_t n, cudaStream_t s)
{
    k_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, v, n);
}

}  // namespace rbx
