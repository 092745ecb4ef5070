// Born forward for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA-graph capture
// that must not add allocation nodes, plug-ins hosted by a framework whose caching
// allocator owns the whole device, or real-time services that forbid allocation after
// start-up. rbx_forward_noalloc serves them: it computes the same D as rbx_forward but
// takes the tables straight from the caller, synthesises the Green's functions inside
// the contraction (no N x X operand buffer), and keeps its only scratch -- the split
// partial sums -- in one fixed array in this library's device memory.
//
// The scratch is a file-scope __device__ array of kScratchElems float2 (8 MiB). Every GPU
// that loads the library holds it until the process exits. All calls share it, and each
// call overwrites every element it later reads, so nothing needs clearing between calls;
// calls whose work overlaps on the GPU (different streams, or different host threads on
// one device) race on it and must be serialised by the caller.
//
// In host code the array's name is only a stand-in for the device object, so the device
// address is fetched with cudaGetSymbolAddress once per device, with that device current,
// on the first call made on it. That first call may load the module; make it before any
// stream capture.
#include "rbx_internal.cuh"

#include <cmath>
#include <cstdio>
#include <mutex>

namespace rbx {

constexpr size_t kScratchElems = 1u << 20;   // float2 elements: 8 MiB
static __device__ __align__(256) float2 g_fwd_scratch[kScratchElems];

namespace {

constexpr int TM = 64, TK = 16;

__device__ __forceinline__ float phase_cycles_na(float T, int K, float fhi, float flo)
{
    float p = fhi * T;
    float err = fmaf(fhi, T, -p) + flo * T;
    float r = (p - rintf(p)) + err;
    return r + 0.125f - 0.25f * (float)K;
}

// G_e[x] = C a exp(i 2 pi (f T - K/4 + 1/8)), 0 where a = 0 (uncovered). Each entry is formed
// once per tile it joins, so the sine and cosine are the hardware ones on the phase taken to
// whole turns ([-pi, pi] rad, absolute error about 4e-7, far inside the FP32 tolerance 1e-5).
__device__ __forceinline__ float2 green_na(const float *T, const float *a, const uint8_t *K, size_t i, float fhi,
                                          float flo, float C)
{
    float av = a[i];
    if (!(av > 0.f)) return make_float2(0.f, 0.f);
    float s, c;
    const float ph = phase_cycles_na(T[i], (int)K[i], fhi, flo);
    __sincosf(6.28318530717958647692f * (ph - rintf(ph)), &s, &c);
    float A = C * av;
    return make_float2(A * c, A * s);
}

__device__ __forceinline__ void cmac_na(float2 &acc, float2 a, float2 b)
{
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// Upper-triangle tile pairs of D = sum_x G_e G_r v, split over the mask nodes; the
// Green's functions are formed from the tables while the tiles are loaded.
__global__ __launch_bounds__(256) void k_forward_tables_noalloc(const float *__restrict__ T, const float *__restrict__ a,
                                                                const uint8_t *__restrict__ K,
                                                                const float *__restrict__ v, int N, int X, int xchunk,
                                                                float fhi, float flo, float C, float2 *__restrict__ part)
{
    int Tn = (N + TM - 1) / TM;
    int b = blockIdx.x, te = 0;
    while (b >= Tn - te) { b -= Tn - te; te++; }
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
        float vv = ok ? v[x] : 0.f;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int row = lr + 16 * q;
            int e = te * TM + row, r = tr * TM + row;
            As[lk][row] = (ok && e < N) ? green_na(T, a, K, (size_t)e * X + x, fhi, flo, C) : make_float2(0.f, 0.f);
            float2 g = (ok && r < N) ? green_na(T, a, K, (size_t)r * X + x, fhi, flo, C) : make_float2(0.f, 0.f);
            Bs[lk][row] = make_float2(g.x * vv, g.y * vv);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; k++) {
            float2 aa[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; i++) aa[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) bb[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) cmac_na(acc[i][j], aa[i], bb[j]);
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

std::mutex g_scratch_mu;
float2 *g_scratch_ptr[64] = {};

void seterr(char *err, size_t errlen, const char *msg)
{
    if (err && errlen) snprintf(err, errlen, "%s", msg);
}

}  // namespace
}  // namespace rbx

using namespace rbx;

extern "C" rbx_status rbx_forward_noalloc(const float *T_dev, const float *a_dev, const uint8_t *K_dev,
                                          const float *v_dev, int n_xducers, int n_nodes, double freq_hz, double c0,
                                          void *D_dev, void *cuda_stream, char *err, size_t errlen)
{
    if (!T_dev || !a_dev || !K_dev || !v_dev || !D_dev) {
        seterr(err, errlen, "null pointer argument");
        return RBX_EINVAL;
    }
    const int N = n_xducers, X = n_nodes;
    if (N < 3 || X < 1 || !(freq_hz > 0) || !std::isfinite(freq_hz) || !(c0 > 0) || !std::isfinite(c0)) {
        seterr(err, errlen, "need n_xducers >= 3, n_nodes >= 1, finite freq_hz > 0 and c0 > 0");
        return RBX_EINVAL;
    }
    if ((size_t)N * (size_t)N > kScratchElems) {
        seterr(err, errlen, "n_xducers exceeds 1024: N*N partial sums must fit the 8 MiB fixed scratch");
        return RBX_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        seterr(err, errlen, "no current CUDA device (or device index >= 64)");
        return RBX_ECUDA;
    }
    float2 *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_fwd_scratch);
            if (e != cudaSuccess || !p) {
                char buf[256];
                snprintf(buf, sizeof buf, "cudaGetSymbolAddress of the forward scratch failed: %s",
                         cudaGetErrorString(e));
                seterr(err, errlen, buf);
                return RBX_ECUDA;
            }
            g_scratch_ptr[dev] = static_cast<float2 *>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    int splits = forward_splits(N, X);
    int cap = (int)(kScratchElems / ((size_t)N * N));
    if (splits > cap) splits = cap;
    int Tn = (N + TM - 1) / TM, pairs = Tn * (Tn + 1) / 2;
    int xchunk = (X + splits - 1) / splits;
    xchunk = (xchunk + TK - 1) / TK * TK;
    splits = (X + xchunk - 1) / xchunk;
    float fhi = (float)freq_hz, flo = (float)(freq_hz - (double)fhi);
    float C = (float)(1.0 / std::sqrt(8.0 * 3.14159265358979323846 * (2.0 * 3.14159265358979323846 * freq_hz) / c0));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    k_forward_tables_noalloc<<<dim3(pairs, splits), 256, 0, s>>>(T_dev, a_dev, K_dev, v_dev, N, X, xchunk, fhi, flo, C,
                                                                 scratch);
    launch_forward_reduce(scratch, N, splits, static_cast<float2 *>(D_dev), s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof buf, "kernel launch failed: %s", cudaGetErrorString(e));
        seterr(err, errlen, buf);
        return RBX_ECUDA;
    }
    seterr(err, errlen, "");
    return RBX_OK;
}
