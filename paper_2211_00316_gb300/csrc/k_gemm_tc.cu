// Steps a6-a8 on the 5th-generation tensor cores (tcgen05, BF16 inputs, FP32 accumulation
// in tensor memory), for the BF16 precision of the library.
//
// Complex operands are kept as planar BF16 (re and im planes, K-major). One complex
// multiply-accumulate is four real MMAs into two accumulators; the -Im*Im term uses the
// instruction descriptor's negate-A bit, so no negated copy is stored:
//   acc_re += A_re B_re^T - A_im B_im^T,   acc_im += A_re B_im^T + A_im B_re^T.
//
// Forward (Eqs. perturb1, derivative): D = G diag(v) G^T, M = e (128), N = r (128),
// K = mask nodes, upper tile pairs only, K split over CTAs, FP32 partials reduced in a
// fixed order (shared with the FP32 path).
// Back-projection (Eq. sound_speed_update2, factorised): for a tile of 128 mask nodes and
// 128 emitters, P0 = U^T R_s and P1 = (conj(kappa) U)^T R_s share the R_s tiles (8 MMAs
// per K step, 4 accumulators = all 512 TMEM columns); the epilogue forms
// sum_e [u_e P0 + s kappa_e u_e P1] per node from tensor memory and the bf16 planes.
//
// Warp roles (192 threads, one CTA per SM): warp 0 issues TMA loads, warp 1 owns tensor
// memory and issues the MMAs from one thread, warps 2-5 drain the accumulators (warp w
// reads TMEM lanes 32 (w mod 4) .. +31).
#include "rbx_internal.cuh"
#include "tc_sm100.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace rbx {
using namespace tc;

namespace {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr uint32_t TILE = BM * BK * 2;        // 16 KB: 128 rows x 64 BF16 (128 B per row)

constexpr int F_STAGES = 3, F_TILES = 4;     // forward: Gre, Gim | Gvre, Gvim
constexpr size_t F_SMEM = 1024 + (size_t)F_STAGES * F_TILES * TILE + 256;
constexpr int B_STAGES = 2, B_TILES = 6;     // back-projection: Ure, Uim, Vre, Vim | Rsre, Rsim
constexpr size_t B_SMEM = 1024 + (size_t)B_STAGES * B_TILES * TILE + 256;

__device__ __forceinline__ float phase_cycles_tc(float T, int K, float fhi, float flo)
{
    float p = fhi * T;
    float err = fmaf(fhi, T, -p) + flo * T;
    float r = (p - rintf(p)) + err;
    return r + 0.125f - 0.25f * (float)K;
}

// sin and cos of 2 pi ph (ph in cycles) for the BF16 operands: the phase taken to whole turns
// ([-1/2, 1/2] cycles, [-pi, pi] rad) and the hardware sine / cosine, whose absolute error
// there (about 4e-7) is far below the planes' resolution (2^-8 BF16, 2^-16 split BF16). Every
// kernel that forms these operands uses it, so they agree bit for bit.
__device__ __forceinline__ void sincos_turns_tc(float ph, float *s, float *c)
{
    const float r = ph - rintf(ph);
    __sincosf(6.28318530717958647692f * r, s, c);
}

// G v with its rounding fixed (no contraction left to the compiler), so every kernel that
// forms the forward operands gives the same bits
__device__ __forceinline__ float gv_re(float gr, float gi, float2 v) { return __fmaf_rn(gr, v.x, -__fmul_rn(gi, v.y)); }
__device__ __forceinline__ float gv_im(float gr, float gi, float2 v) { return __fmaf_rn(gr, v.y, __fmul_rn(gi, v.x)); }

__device__ __forceinline__ uint8_t *align1024(uint8_t *p)
{
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

// ---------------------------------------------------------------- forward

// Operand maps of one K pass: A (re, im) and B (re, im).
struct Maps4 {
    CUtensorMap are, aim, bre, bim;
};

// passes = 1: A_hi B_hi. passes = 3 (split BF16): A_hi B_hi + A_hi B_lo + A_lo B_hi.
// With split BF16 the tensor-memory accumulators are drained every kSeg K chunks into the
// CTA's FP32 partial tile in global memory (the CTA owns that tile), so no accumulation in
// tensor memory runs over more than kSeg x 64 mask nodes (its long-K rounding would
// otherwise exceed the split's own error); two accumulator buffers alternate so the MMAs
// never wait for the drain. Plain BF16, whose error is its input rounding, uses one segment.
constexpr int kSeg = 16;

__global__ __launch_bounds__(192, 1) void k_forward_tc(const __grid_constant__ Maps4 hi, const __grid_constant__ Maps4 lo,
                                                       int passes, int N, int ntile, int nk, int kper,
                                                       float2 *__restrict__ part, unsigned *__restrict__ err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *tiles = align1024(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + (size_t)F_STAGES * F_TILES * TILE);
    uint64_t *empty = full + F_STAGES;
    uint64_t *accf = empty + F_STAGES;     // [2] accumulator buffer ready to drain
    uint64_t *acce = accf + 2;             // [2] accumulator buffer drained
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acce + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    int b = blockIdx.x, te = 0;
    while (b >= ntile - te) { b -= ntile - te; te++; }
    const int tr = te + b;
    const int split = blockIdx.y;
    const int c0 = split * kper, nc = min(nk, c0 + kper) - c0;
    const int ntot = passes * nc;
    const int seglen = passes == 3 ? kSeg : (ntot > 0 ? ntot : 1);
    const int nseg = (ntot + seglen - 1) / seglen;

    if (threadIdx.x == 0) {
        for (int s = 0; s < F_STAGES; s++) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
        for (int q = 0; q < 2; q++) { mbar_init(accf + q, 1); mbar_init(acce + q, 128); }
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tslot, 512);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        prefetch_tmap(&hi.are); prefetch_tmap(&hi.aim); prefetch_tmap(&hi.bre); prefetch_tmap(&hi.bim);
        int issued = 0;
        for (int c = 0; c < ntot; c++) {
            int s = c % F_STAGES;
            if (c >= F_STAGES && !mbar_wait(empty + s, ((c / F_STAGES) - 1) & 1)) { atomicOr(err, 1u); break; }
            mbar_arrive_expect_tx(full + s, F_TILES * TILE);
            uint32_t base = smem_u32(tiles + (size_t)s * F_TILES * TILE);
            const int pass = c / nc;
            const Maps4 &A = pass == 2 ? lo : hi, &B = pass == 1 ? lo : hi;
            int kx = (c0 + c - pass * nc) * BK;
            tma_load_2d(base, &A.are, full + s, kx, te * BM);
            tma_load_2d(base + TILE, &A.aim, full + s, kx, te * BM);
            tma_load_2d(base + 2 * TILE, &B.bre, full + s, kx, tr * BN);
            tma_load_2d(base + 3 * TILE, &B.bim, full + s, kx, tr * BN);
            issued++;
        }
        // no copy may still be in flight when the CTA retires
        for (int c = (issued > F_STAGES ? issued - F_STAGES : 0); c < issued; c++)
            if (!mbar_wait(full + (c % F_STAGES), (c / F_STAGES) & 1)) atomicOr(err, 4u);
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t ip = idesc_bf16(BM, BN, 0), in = idesc_bf16(BM, BN, 1);
            bool ok = true;
            for (int c = 0; c < ntot && ok; c++) {
                const int seg = c / seglen, cs = c - seg * seglen, buf = seg & 1;
                if (cs == 0 && seg >= 2) {
                    if (!mbar_wait(acce + buf, ((seg >> 1) - 1) & 1)) { atomicOr(err, 32u); ok = false; break; }
                    fence_after();
                }
                const uint32_t dre = tmem + buf * 2 * BN, dim = dre + BN;
                int s = c % F_STAGES;
                if (!mbar_wait(full + s, (c / F_STAGES) & 1)) { atomicOr(err, 2u); ok = false; break; }
                fence_after();
                uint32_t base = smem_u32(tiles + (size_t)s * F_TILES * TILE);
#pragma unroll
                for (int k = 0; k < BK / 16; k++) {
                    uint64_t a0 = desc_sw128(base + k * 32), a1 = desc_sw128(base + TILE + k * 32);
                    uint64_t b0 = desc_sw128(base + 2 * TILE + k * 32), b1 = desc_sw128(base + 3 * TILE + k * 32);
                    uint32_t acc = (cs > 0 || k > 0) ? 1u : 0u;
                    mma_bf16(dre, a0, b0, ip, acc);
                    mma_bf16(dre, a1, b1, in, 1u);
                    mma_bf16(dim, a0, b1, ip, acc);
                    mma_bf16(dim, a1, b0, ip, 1u);
                }
                mma_commit(empty + s);
                if (cs == seglen - 1 || c == ntot - 1) mma_commit(accf + buf);
            }
            // every MMA of this CTA has completed once the last buffer is signalled
            if (ntot > 0 && !mbar_wait(accf + ((nseg - 1) & 1), ((nseg - 1) >> 1) & 1)) atomicOr(err, 8u);
        }
        __syncwarp();
    } else if (warp >= 2) {
        const int sub = warp & 3, row = sub * 32 + lane;
        const int e = te * BM + row;
        float2 *P = part + (size_t)split * N * N + (size_t)e * N;
        const uint32_t lanes = (uint32_t)(sub * 32) << 16;
        for (int sg = 0; sg < nseg; sg++) {
            const int buf = sg & 1;
            bool ok = __all_sync(0xffffffffu, mbar_wait(accf + buf, (sg >> 1) & 1));
            fence_after();
            if (!ok) {
                if (lane == 0) atomicOr(err, 16u);
                break;
            }
            const uint32_t dre = tmem + buf * 2 * BN;
#pragma unroll 1
            for (int cc = 0; cc < BN; cc += 32) {
                float vr[32], vi[32];
                tmem_ld32(tmem + lanes + (dre - tmem) + cc, vr);
                tmem_ld32(tmem + lanes + (dre - tmem) + BN + cc, vi);
                if (e < N) {
#pragma unroll
                    for (int i = 0; i < 32; i++) {
                        int r = tr * BN + cc + i;
                        if (r < N) {
                            float2 v = make_float2(vr[i], vi[i]);
                            if (sg > 0) {
                                float2 o = P[r];
                                v.x += o.x;
                                v.y += o.y;
                            }
                            P[r] = v;
                        }
                    }
                }
            }
            fence_before();
            mbar_arrive(acce + buf);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// Fused-synthesis candidate of the plain BF16 forward (the tuner times it against the
// separate synthesis pass plus k_forward_tc and keeps the faster): no operand planes. The
// four epilogue warps, idle during the K loop of the plain forward (one accumulation
// segment), form each stage's tiles from the tables themselves: G_e[x] for the 128 emitter
// rows of the tile pair and G_r[x] v[x] for its 128 receiver rows (Eqs. 2D_greens, perturb1),
// with the same phase, sine/cosine and rounding to BF16 as the synthesis pass, so D is the same
// bit for bit. They store the values in the 128-byte-swizzled K-major layout the MMA
// descriptors read (row r at 128 r bytes, its 16-byte chunk c at chunk c ^ (r mod 8)), make the
// generic-proxy writes visible to the tensor cores' async proxy, and arrive on the stage's
// barrier. Each table entry is formed once per tile pair it belongs to (N / 128 times), where
// the separate pass forms it once and TMA streams the BF16 planes.
__global__ __launch_bounds__(192, 1) void k_forward_tc_fused(const TabEntry *__restrict__ tab,
                                                             const float2 *__restrict__ v, int N, int X, int ntile,
                                                             int nk, int kper, float fhi, float flo, float C,
                                                             float2 *__restrict__ part, unsigned *__restrict__ err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *tiles = align1024(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + (size_t)F_STAGES * F_TILES * TILE);
    uint64_t *empty = full + F_STAGES;
    uint64_t *accf = empty + F_STAGES;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(accf + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    int b = blockIdx.x, te = 0;
    while (b >= ntile - te) { b -= ntile - te; te++; }
    const int tr = te + b;
    const int split = blockIdx.y;
    const int c0 = split * kper, nc = min(nk, c0 + kper) - c0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < F_STAGES; s++) { mbar_init(full + s, 128); mbar_init(empty + s, 1); }
        mbar_init(accf, 1);
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tslot, 512);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 1) {
        if (lane == 0) {
            const uint32_t ip = idesc_bf16(BM, BN, 0), in = idesc_bf16(BM, BN, 1);
            const uint32_t dre = tmem, dim = tmem + BN;
            bool ok = true;
            for (int c = 0; c < nc && ok; c++) {
                const int s = c % F_STAGES;
                if (!mbar_wait(full + s, (c / F_STAGES) & 1)) { atomicOr(err, 2u); ok = false; break; }
                fence_after();
                const uint32_t base = smem_u32(tiles + (size_t)s * F_TILES * TILE);
#pragma unroll
                for (int k = 0; k < BK / 16; k++) {
                    uint64_t a0 = desc_sw128(base + k * 32), a1 = desc_sw128(base + TILE + k * 32);
                    uint64_t b0 = desc_sw128(base + 2 * TILE + k * 32), b1 = desc_sw128(base + 3 * TILE + k * 32);
                    uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
                    mma_bf16(dre, a0, b0, ip, acc);
                    mma_bf16(dre, a1, b1, in, 1u);
                    mma_bf16(dim, a0, b1, ip, acc);
                    mma_bf16(dim, a1, b0, ip, 1u);
                }
                mma_commit(empty + s);
            }
            if (nc > 0) mma_commit(accf);
            if (nc > 0 && !mbar_wait(accf, 0)) atomicOr(err, 8u);
        }
        __syncwarp();
    } else if (warp >= 2) {
        // producers: warp w forms tile rows 32 (w - 2) .. +31 of both operands
        const int pw = warp - 2;
        bool ok = true;
        for (int c = 0; c < nc && ok; c++) {
            const int s = c % F_STAGES;
            if (c >= F_STAGES) {
                ok = __all_sync(0xffffffffu, mbar_wait(empty + s, ((c / F_STAGES) - 1) & 1));
                if (!ok) {
                    if (lane == 0) atomicOr(err, 1u);
                    break;
                }
            }
            uint8_t *base = tiles + (size_t)s * F_TILES * TILE;
            const int kx = (c0 + c) * BK;
            float2 vv[2];
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int x = kx + lane + 32 * q;
                vv[q] = x < X ? v[x] : make_float2(0.f, 0.f);
            }
#pragma unroll 1
            for (int rr = 0; rr < 32; rr++) {
                const int r = pw * 32 + rr;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int row = (h ? tr : te) * BM + r;
#pragma unroll
                    for (int q = 0; q < 2; q++) {
                        const int col = lane + 32 * q, x = kx + col;
                        float gr = 0.f, gi = 0.f;
                        if (row < N && x < X) {
                            const TabEntry t = tab[(size_t)row * X + x];
                            if (t.idk != kUncovered) {
                                float sn, cs;
                                sincos_turns_tc(phase_cycles_tc(t.T, (int)(t.idk & 0xffu), fhi, flo), &sn, &cs);
                                gr = C * t.a * cs;
                                gi = C * t.a * sn;
                            }
                        }
                        const float re = h ? gv_re(gr, gi, vv[q]) : gr, im = h ? gv_im(gr, gi, vv[q]) : gi;
                        const uint32_t off = (uint32_t)r * 128u + ((((uint32_t)col >> 3) ^ ((uint32_t)r & 7u)) << 4) +
                                             (((uint32_t)col & 7u) << 1);
                        *reinterpret_cast<__nv_bfloat16 *>(base + (2 * h) * TILE + off) = __float2bfloat16_rn(re);
                        *reinterpret_cast<__nv_bfloat16 *>(base + (2 * h + 1) * TILE + off) = __float2bfloat16_rn(im);
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(full + s);
        }
        // epilogue: the single accumulation segment into the CTA's partial tile
        const int sub = warp & 3, row = sub * 32 + lane;
        const int e = te * BM + row;
        float2 *P = part + (size_t)split * N * N + (size_t)e * N;
        const uint32_t lanes = (uint32_t)(sub * 32) << 16;
        if (ok && nc > 0) {
            ok = __all_sync(0xffffffffu, mbar_wait(accf, 0));
            fence_after();
            if (!ok && lane == 0) atomicOr(err, 16u);
        }
        if (ok) {
#pragma unroll 1
            for (int cc = 0; cc < BN; cc += 32) {
                float vr[32], vi[32];
                if (nc > 0) {
                    tmem_ld32(tmem + lanes + cc, vr);
                    tmem_ld32(tmem + lanes + BN + cc, vi);
                } else {
#pragma unroll
                    for (int i = 0; i < 32; i++) vr[i] = vi[i] = 0.f;
                }
                if (e < N) {
#pragma unroll
                    for (int i = 0; i < 32; i++) {
                        const int r = tr * BN + cc + i;
                        if (r < N) P[r] = make_float2(vr[i], vi[i]);
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------- back-projection

// Operand maps of one K pass: A = u and conj(kappa) u (re, im), B = R_s (re, im).
struct Maps6 {
    CUtensorMap ure, uim, vre, vim, rre, rim;
};

// passes = 1: A_hi B_hi; passes = 3 (split BF16) adds A_hi B_lo and A_lo B_hi, and the
// epilogue weights are read as hi + lo. With split BF16, as in the forward, no accumulation in
// tensor memory runs over more than kSeg K chunks: the MMAs pause at each segment's end while
// the epilogue adds that segment's row-dot into its registers (the row-dot is linear in P),
// then restart from zero (one accumulator set, so the pause is not hidden; split BF16 only).
template <bool SPLIT>
__global__ __launch_bounds__(192, 1) void k_backproject_tc(const __grid_constant__ Maps6 hi,
                                                           const __grid_constant__ Maps6 lo,
                                                           const __nv_bfloat16 *__restrict__ planes, size_t pstride,
                                                           int Npad, int nk, float sgn, float2 *__restrict__ bpart,
                                                           int Xp, unsigned *__restrict__ err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *tiles = align1024(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + (size_t)B_STAGES * B_TILES * TILE);
    uint64_t *empty = full + B_STAGES;
    uint64_t *accb = empty + B_STAGES;     // accumulators of a segment ready to drain
    uint64_t *accd = accb + 1;             // accumulators drained
    uint32_t *tslot = reinterpret_cast<uint32_t *>(accd + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int et = blockIdx.x, xt = blockIdx.y;
    constexpr int passes = SPLIT ? 3 : 1;
    const int ntot = passes * nk;
    const int seglen = SPLIT ? kSeg : ntot;
    const int nseg = SPLIT ? (ntot + kSeg - 1) / kSeg : 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < B_STAGES; s++) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
        mbar_init(accb, 1);
        mbar_init(accd, 128);
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tslot, 512);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        prefetch_tmap(&hi.ure); prefetch_tmap(&hi.uim); prefetch_tmap(&hi.vre); prefetch_tmap(&hi.vim);
        prefetch_tmap(&hi.rre); prefetch_tmap(&hi.rim);
        int issued = 0;
        for (int c = 0; c < ntot; c++) {
            int s = c % B_STAGES;
            if (c >= B_STAGES && !mbar_wait(empty + s, ((c / B_STAGES) - 1) & 1)) { atomicOr(err, 1u); break; }
            mbar_arrive_expect_tx(full + s, B_TILES * TILE);
            uint32_t base = smem_u32(tiles + (size_t)s * B_TILES * TILE);
            const int pass = c / nk;
            const Maps6 &A = pass == 2 ? lo : hi, &B = pass == 1 ? lo : hi;
            int kx = (c - pass * nk) * BK;
            tma_load_2d(base, &A.ure, full + s, kx, xt * BM);
            tma_load_2d(base + TILE, &A.uim, full + s, kx, xt * BM);
            tma_load_2d(base + 2 * TILE, &A.vre, full + s, kx, xt * BM);
            tma_load_2d(base + 3 * TILE, &A.vim, full + s, kx, xt * BM);
            tma_load_2d(base + 4 * TILE, &B.rre, full + s, kx, et * BN);
            tma_load_2d(base + 5 * TILE, &B.rim, full + s, kx, et * BN);
            issued++;
        }
        for (int c = (issued > B_STAGES ? issued - B_STAGES : 0); c < issued; c++)
            if (!mbar_wait(full + (c % B_STAGES), (c / B_STAGES) & 1)) atomicOr(err, 4u);
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t ip = idesc_bf16(BM, BN, 0), in = idesc_bf16(BM, BN, 1);
            const uint32_t p0r = tmem, p0i = tmem + BN, p1r = tmem + 2 * BN, p1i = tmem + 3 * BN;
            for (int c = 0; c < ntot; c++) {
                const int seg = SPLIT ? c / kSeg : 0, cs = c - seg * seglen;
                if (cs == 0 && seg >= 1) {   // the previous segment's accumulators have been read
                    if (!mbar_wait(accd, (seg - 1) & 1)) { atomicOr(err, 32u); break; }
                    fence_after();
                }
                int s = c % B_STAGES;
                if (!mbar_wait(full + s, (c / B_STAGES) & 1)) { atomicOr(err, 2u); break; }
                fence_after();
                uint32_t base = smem_u32(tiles + (size_t)s * B_TILES * TILE);
#pragma unroll
                for (int k = 0; k < BK / 16; k++) {
                    uint64_t ur = desc_sw128(base + k * 32), ui = desc_sw128(base + TILE + k * 32);
                    uint64_t vr = desc_sw128(base + 2 * TILE + k * 32), vi = desc_sw128(base + 3 * TILE + k * 32);
                    uint64_t rr = desc_sw128(base + 4 * TILE + k * 32), ri = desc_sw128(base + 5 * TILE + k * 32);
                    uint32_t acc = (cs > 0 || k > 0) ? 1u : 0u;
                    mma_bf16(p0r, ur, rr, ip, acc);
                    mma_bf16(p0r, ui, ri, in, 1u);
                    mma_bf16(p0i, ur, ri, ip, acc);
                    mma_bf16(p0i, ui, rr, ip, 1u);
                    mma_bf16(p1r, vr, rr, ip, acc);
                    mma_bf16(p1r, vi, ri, in, 1u);
                    mma_bf16(p1i, vr, ri, ip, acc);
                    mma_bf16(p1i, vi, rr, ip, 1u);
                }
                mma_commit(empty + s);
                if (cs == seglen - 1 || c == ntot - 1) mma_commit(accb);
            }
            // every MMA of this CTA has completed once the last segment is signalled
            if (!mbar_wait(accb, (nseg - 1) & 1)) atomicOr(err, 8u);
        }
        __syncwarp();
    } else if (warp >= 2) {
        const int sub = warp & 3, row = sub * 32 + lane;
        const int x = xt * BM + row;
        float gre = 0.f, gim = 0.f;
        bool ok = true;
        for (int sg = 0; sg < nseg && ok; sg++) {
            ok = __all_sync(0xffffffffu, mbar_wait(accb, sg & 1));
            fence_after();
            if (!ok) break;
            const uint32_t lanes = (uint32_t)(sub * 32) << 16;
            // epilogue weights at [x][e]: u (planes 0, 1) and kappa u (planes 4, 5); with
            // split BF16 the lo parts are planes 6 + (0, 1, 4, 5)
            const __nv_bfloat16 *w0r = planes + (size_t)x * Npad + et * BN;
            const __nv_bfloat16 *w0i = w0r + pstride, *w1r = w0r + 4 * pstride, *w1i = w0r + 5 * pstride;
            const size_t lo_off = 6 * pstride;
#pragma unroll 1
            for (int cc = 0; cc < BN; cc += 32) {
                float a0r[32], a0i[32], a1r[32], a1i[32];
                tmem_ld32(tmem + lanes + cc, a0r);
                tmem_ld32(tmem + lanes + BN + cc, a0i);
                tmem_ld32(tmem + lanes + 2 * BN + cc, a1r);
                tmem_ld32(tmem + lanes + 3 * BN + cc, a1i);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    uint4 r0 = *reinterpret_cast<const uint4 *>(w0r + cc + 8 * q);
                    uint4 i0 = *reinterpret_cast<const uint4 *>(w0i + cc + 8 * q);
                    uint4 r1 = *reinterpret_cast<const uint4 *>(w1r + cc + 8 * q);
                    uint4 i1 = *reinterpret_cast<const uint4 *>(w1i + cc + 8 * q);
                    uint4 r0l = make_uint4(0, 0, 0, 0), i0l = r0l, r1l = r0l, i1l = r0l;
                    if (passes == 3) {
                        r0l = *reinterpret_cast<const uint4 *>(w0r + lo_off + cc + 8 * q);
                        i0l = *reinterpret_cast<const uint4 *>(w0i + lo_off + cc + 8 * q);
                        r1l = *reinterpret_cast<const uint4 *>(w1r + lo_off + cc + 8 * q);
                        i1l = *reinterpret_cast<const uint4 *>(w1i + lo_off + cc + 8 * q);
                    }
                    const __nv_bfloat162 *R0 = reinterpret_cast<const __nv_bfloat162 *>(&r0);
                    const __nv_bfloat162 *I0 = reinterpret_cast<const __nv_bfloat162 *>(&i0);
                    const __nv_bfloat162 *R1 = reinterpret_cast<const __nv_bfloat162 *>(&r1);
                    const __nv_bfloat162 *I1 = reinterpret_cast<const __nv_bfloat162 *>(&i1);
                    const __nv_bfloat162 *R0l = reinterpret_cast<const __nv_bfloat162 *>(&r0l);
                    const __nv_bfloat162 *I0l = reinterpret_cast<const __nv_bfloat162 *>(&i0l);
                    const __nv_bfloat162 *R1l = reinterpret_cast<const __nv_bfloat162 *>(&r1l);
                    const __nv_bfloat162 *I1l = reinterpret_cast<const __nv_bfloat162 *>(&i1l);
#pragma unroll
                    for (int h = 0; h < 4; h++) {
                        float2 wr0 = __bfloat1622float2(R0[h]), wi0 = __bfloat1622float2(I0[h]);
                        float2 wr1 = __bfloat1622float2(R1[h]), wi1 = __bfloat1622float2(I1[h]);
                        float2 t;
                        t = __bfloat1622float2(R0l[h]); wr0.x += t.x; wr0.y += t.y;
                        t = __bfloat1622float2(I0l[h]); wi0.x += t.x; wi0.y += t.y;
                        t = __bfloat1622float2(R1l[h]); wr1.x += t.x; wr1.y += t.y;
                        t = __bfloat1622float2(I1l[h]); wi1.x += t.x; wi1.y += t.y;
                        int j = 8 * q + 2 * h;
                        gre += wr0.x * a0r[j] - wi0.x * a0i[j] + sgn * (wr1.x * a1r[j] - wi1.x * a1i[j]);
                        gim += wr0.x * a0i[j] + wi0.x * a0r[j] + sgn * (wr1.x * a1i[j] + wi1.x * a1r[j]);
                        gre += wr0.y * a0r[j + 1] - wi0.y * a0i[j + 1] + sgn * (wr1.y * a1r[j + 1] - wi1.y * a1i[j + 1]);
                        gim += wr0.y * a0i[j + 1] + wi0.y * a0r[j + 1] + sgn * (wr1.y * a1i[j + 1] + wi1.y * a1r[j + 1]);
                    }
                }
            }
            fence_before();
            mbar_arrive(accd);
        }
        if (ok)
            bpart[(size_t)et * Xp + x] = make_float2(gre, gim);
        else if (lane == 0)
            atomicOr(err, 16u);
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------- operand synthesis

// value = hi + lo with hi = bf16(value), lo = bf16(value - hi) (split BF16)
__device__ __forceinline__ void put_split(__nv_bfloat16 *hi, __nv_bfloat16 *lo, float v)
{
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    *hi = h;
    if (lo) *lo = __float2bfloat16_rn(v - __bfloat162float(h));
}


// planes [4][Npad][Xpad]: Gre, Gim, (G v)re, (G v)im (then 4 lo planes when split);
// G_e[x] = C a exp(i 2 pi (f T - K/4 + 1/8))
__global__ void k_synth_fwd_tc(const TabEntry *__restrict__ tab, const float2 *__restrict__ v, int N, int X, int Xpad,
                               size_t pstride, float fhi, float flo, float C, __nv_bfloat16 *__restrict__ planes,
                               int split)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)N * X) return;
    int e = (int)(i / X), x = (int)(i % X);
    TabEntry t = tab[i];
    float gr = 0.f, gi = 0.f;
    if (t.idk != kUncovered) {
        float s, c;
        sincos_turns_tc(phase_cycles_tc(t.T, (int)(t.idk & 0xffu), fhi, flo), &s, &c);
        gr = C * t.a * c;
        gi = C * t.a * s;
    }
    const float2 vv = v[x];
    size_t o = (size_t)e * Xpad + x;
    __nv_bfloat16 *lo = split ? planes + 4 * pstride : nullptr;
    put_split(planes + o, lo ? lo + o : nullptr, gr);
    put_split(planes + pstride + o, lo ? lo + pstride + o : nullptr, gi);
    put_split(planes + 2 * pstride + o, lo ? lo + 2 * pstride + o : nullptr, gv_re(gr, gi, vv));
    put_split(planes + 3 * pstride + o, lo ? lo + 3 * pstride + o : nullptr, gv_im(gr, gi, vv));
}

// 16-byte asynchronous copy global -> shared (L2 only), and its group fences.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// One synthesis tile: 32 nodes x 32 transducers, with a halo row of transducers on each side.
constexpr int kSynSlots = 34 * 32;   // slot s holds row (e0 - 1 + s) mod N, nodes x0 .. x0 + 31

// Queue the copies of tile t's table entries into buf (entries past the last node are not
// copied; the consumer treats them as uncovered).
__device__ __forceinline__ void synth_tile_load(const TabEntry *__restrict__ tab, int N, int X, int XT, int t,
                                                TabEntry *buf)
{
    const int ET = (N + 31) / 32, x0 = (t / ET) * 32, e0 = (t % ET) * 32;
    for (int idx = threadIdx.x; idx < kSynSlots; idx += 256) {
        const int slot = idx >> 5, x = x0 + (idx & 31);
        if (x < X) {
            const int e = (e0 - 1 + slot + N) % N;
            cp_async16(buf + idx, tab + (size_t)e * X + x);
        }
    }
}

// planes [6][Xp][Npad] at [x][e]: u, conj(kappa) u, kappa u (re, im each);
// u_e[x] = dgamma / (C a) exp(-i 2 pi (f T - K/4 + 1/8)), kappa = exp(i gamma).
// The angular density dgamma (step a4) is formed here from the direction angles of the
// neighbouring transducers: a 32-transducer tile reads one halo row on each side (rows wrap
// around the ring), so the tables are read once more by 1/16 instead of a separate pass.
// With FWD the same pass also writes the forward's planes (those of k_synth_fwd_tc, from the
// same phase): an update reads its tables once for both contractions' operands.
// Persistent: each block walks the tiles t = blockIdx.x, + gridDim.x, ... (transducer blocks
// fastest, so that the blocks running at once complete whole [x][e] rows of the
// back-projection planes, 8 % faster than nodes fastest) with
// two shared-memory buffers, the next tile's entries copied in while the current one is
// formed and stored, so that table reads stay in flight between the blocks' barriers.
template <bool FWD, bool SPLIT>
__global__ __launch_bounds__(256, SPLIT ? 3 : 4) void k_synth_tc(const TabEntry *__restrict__ tab, int N, int X, int Npad,
                                                     size_t pstride, float fhi, float flo, float C,
                                                     __nv_bfloat16 *__restrict__ planes, const float2 *__restrict__ bw,
                                                     int Xpad, size_t fpstride, __nv_bfloat16 *__restrict__ fplanes,
                                                     int XT, int ntiles)
{
    constexpr int NPL = SPLIT ? 12 : 6;                      // back-projection planes (hi, then lo)
    extern __shared__ __align__(16) unsigned char syn_smem[];
    TabEntry *buf = reinterpret_cast<TabEntry *>(syn_smem);  // [2][kSynSlots]
    // [plane][x][e]: rows of 17 words, the tile transposed and rounded to BF16
    __nv_bfloat16(*sv)[32][34] = reinterpret_cast<__nv_bfloat16(*)[32][34]>(syn_smem + 2 * kSynSlots * sizeof(TabEntry));
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    int t = blockIdx.x, b = 0;
    if (t < ntiles) synth_tile_load(tab, N, X, XT, t, buf);
    cp_async_commit();
    for (; t < ntiles; t += gridDim.x, b ^= 1) {
        if (t + (int)gridDim.x < ntiles) synth_tile_load(tab, N, X, XT, t + gridDim.x, buf + (b ^ 1) * kSynSlots);
        cp_async_commit();
        cp_async_wait1();   // this thread's copies of tile t have landed
        __syncthreads();    // and every thread's
        const TabEntry *B = buf + b * kSynSlots;
        const int ET = (N + 31) / 32, x0 = (t / ET) * 32, e0 = (t % ET) * 32;
        const int x = x0 + tx;
        const bool xin = x < X;
        float2 vv = make_float2(0.f, 0.f);
        if (FWD && xin) vv = bw[x];   // Born weights of node x
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int q = ty + 8 * k;
            float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float gr = 0.f, gi = 0.f;
            const TabEntry r = B[(q + 1) * 32 + tx];   // row e0 + q
            if (xin && e0 + q < N && r.idk != kUncovered) {
                // slot q + 2 is row (e + 1) mod N and slot q row (e - 1) mod N, also for e = 0, N - 1
                const TabEntry &rp = B[(q + 2) * 32 + tx], &rm = B[q * 32 + tx];
                const float dg = (rp.idk != kUncovered && rm.idk != kUncovered) ? dgamma_of(rp.gam, rm.gam) : 0.f;
                // kappa from the hardware sine / cosine (gamma lies in [-pi, pi], absolute error
                // ~1e-6, far below the BF16 planes' and the split planes' 2^-16 resolution)
                float sn, cs, sgm, cgm;
                sincos_turns_tc(phase_cycles_tc(r.T, (int)(r.idk & 0xffu), fhi, flo), &sn, &cs);
                __sincosf(r.gam, &sgm, &cgm);
                const float A = dg * rcp_nr(C * r.a);
                gr = C * r.a * cs;
                gi = C * r.a * sn;
                float ur = A * cs, ui = -A * sn;
                v[0] = ur; v[1] = ui;
                v[2] = cgm * ur + sgm * ui; v[3] = cgm * ui - sgm * ur;   // conj(kappa) u
                v[4] = cgm * ur - sgm * ui; v[5] = cgm * ui + sgm * ur;   // kappa u
            }
#pragma unroll
            for (int m = 0; m < 6; m++) {
                const __nv_bfloat16 h = __float2bfloat16_rn(v[m]);
                sv[m][tx][q] = h;
                if (SPLIT) sv[6 + m][tx][q] = __float2bfloat16_rn(v[m] - __bfloat162float(h));
            }
            if (FWD && e0 + q < N && xin) {
                // G and G v at [e][x], as k_synth_fwd_tc
                const size_t o = (size_t)(e0 + q) * Xpad + x;
                __nv_bfloat16 *lo = SPLIT ? fplanes + 4 * fpstride : nullptr;
                put_split(fplanes + o, SPLIT ? lo + o : nullptr, gr);
                put_split(fplanes + fpstride + o, SPLIT ? lo + fpstride + o : nullptr, gi);
                put_split(fplanes + 2 * fpstride + o, SPLIT ? lo + 2 * fpstride + o : nullptr, gv_re(gr, gi, vv));
                put_split(fplanes + 3 * fpstride + o, SPLIT ? lo + 3 * fpstride + o : nullptr, gv_im(gr, gi, vv));
            }
        }
        __syncthreads();   // the tile is in sv, and buffer b is free for the tile after next
        // write-out: two neighbouring transducers per 32-bit store (Npad, e0 and the planes'
        // base are even, so every store is aligned); entries past the last transducer are
        // zero, as the padding must be
        const uint32_t *sw = reinterpret_cast<const uint32_t *>(&sv[0][0][0]);
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const int item = threadIdx.x + 256 * j, xr = item >> 4, pr = item & 15;
            if (x0 + xr < X) {
                const size_t o = (size_t)(x0 + xr) * Npad + e0 + 2 * pr;
#pragma unroll
                for (int m = 0; m < NPL; m++)
                    *reinterpret_cast<uint32_t *>(planes + m * pstride + o) = sw[(m * 32 + xr) * 17 + pr];
            }
        }
    }
    cp_async_wait0();
}

// R_s (complex N x N) -> planes [2][Npad][Npad] (then 2 lo planes when split)
__global__ void k_rs_planes(const float2 *__restrict__ Rs, int N, int Npad, __nv_bfloat16 *__restrict__ planes,
                            int split)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)N * N) return;
    int e = (int)(i / N), r = (int)(i % N);
    float2 v = Rs[i];
    size_t o = (size_t)e * Npad + r, P = (size_t)Npad * Npad;
    put_split(planes + o, split ? planes + 2 * P + o : nullptr, v.x);
    put_split(planes + P + o, split ? planes + 3 * P + o : nullptr, v.y);
}

// gpart[0][x] = sum over emitter tiles (fixed order); gpart[1][x] = 0 (the stacks are
// already combined with their sign in the epilogue)
__global__ void k_bp_reduce(const float2 *__restrict__ bpart, int ET, int Xp, int X, float2 *__restrict__ gpart)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= X) return;
    float2 s = make_float2(0.f, 0.f);
    for (int t = 0; t < ET; t++) {
        float2 p = bpart[(size_t)t * Xp + x];
        s.x += p.x;
        s.y += p.y;
    }
    gpart[x] = s;
    gpart[(size_t)X + x] = make_float2(0.f, 0.f);
}

// ---------------------------------------------------------------- host helpers

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// BF16 matrix [rows][cols] (cols contiguous, K-major) read in 128-row x 64-column boxes
bool make_map(CUtensorMap *m, const void *base, size_t rows, size_t cols)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// ---------------------------------------------------------------- API used by rbx_api.cu

bool tc_setup(TcPlanes &p, int N, int X, bool split, cudaStream_t st)
{
    p.split = split;
    const int mult = split ? 2 : 1;
    p.N = N;
    p.X = X;
    p.Npad = (N + BM - 1) / BM * BM;
    p.Xpad = (X + BK - 1) / BK * BK;
    p.Xp = (X + BM - 1) / BM * BM;
    p.fwd_pstride = (size_t)p.Npad * p.Xpad;
    p.bp_pstride = (size_t)p.Xp * p.Npad;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p.sms = sms;
    int T = p.Npad / BM, pairs = T * (T + 1) / 2;
    int nk = p.Xpad / BK;
    int splits = pairs >= sms ? 1 : sms / pairs;
    if (splits > nk) splits = nk;
    int kper = (nk + splits - 1) / splits;
    p.fwd_kper = kper;
    p.fwd_splits = (nk + kper - 1) / kper;
    // the autotuner may go up to 4x the heuristic's split (at most one K chunk per CTA)
    const int smax = std::min(nk, std::max(4 * splits, 1));
    p.fwd_max_splits = (nk + (nk + smax - 1) / smax - 1) / ((nk + smax - 1) / smax);
    const size_t fbytes = mult * 4 * p.fwd_pstride * sizeof(__nv_bfloat16);
    const size_t bbytes = mult * 6 * p.bp_pstride * sizeof(__nv_bfloat16);
    const size_t rbytes = mult * 2 * (size_t)p.Npad * p.Npad * sizeof(__nv_bfloat16);
    if (cudaMallocAsync(&p.fplanes, fbytes, st) != cudaSuccess) return false;
    if (cudaMallocAsync(&p.bplanes, bbytes, st) != cudaSuccess) return false;
    if (cudaMallocAsync(&p.rsplanes, rbytes, st) != cudaSuccess) return false;
    if (cudaMallocAsync(reinterpret_cast<void **>(&p.bpart), (size_t)(p.Npad / BN) * p.Xp * sizeof(float2), st) !=
        cudaSuccess)
        return false;
    if (cudaMallocAsync(reinterpret_cast<void **>(&p.err), sizeof(unsigned), st) != cudaSuccess) return false;
    cudaMemsetAsync(p.fplanes, 0, fbytes, st);
    cudaMemsetAsync(p.bplanes, 0, bbytes, st);
    cudaMemsetAsync(p.rsplanes, 0, rbytes, st);
    cudaMemsetAsync(p.err, 0, sizeof(unsigned), st);
    const __nv_bfloat16 *f = static_cast<const __nv_bfloat16 *>(p.fplanes);
    const __nv_bfloat16 *b = static_cast<const __nv_bfloat16 *>(p.bplanes);
    const __nv_bfloat16 *r = static_cast<const __nv_bfloat16 *>(p.rsplanes);
    const size_t P = (size_t)p.Npad * p.Npad;
    bool ok = true;
    for (int h = 0; h < mult; h++) {
        const __nv_bfloat16 *fh = f + (size_t)h * 4 * p.fwd_pstride, *bh = b + (size_t)h * 6 * p.bp_pstride,
                            *rh = r + (size_t)h * 2 * P;
        for (int k = 0; k < 4; k++) ok = ok && make_map(&p.fmaps[h][k], fh + k * p.fwd_pstride, p.Npad, p.Xpad);
        for (int k = 0; k < 4; k++) ok = ok && make_map(&p.bmaps[h][k], bh + k * p.bp_pstride, p.Xp, p.Npad);
        for (int k = 0; k < 2; k++) ok = ok && make_map(&p.bmaps[h][4 + k], rh + (size_t)k * P, p.Npad, p.Npad);
    }
    if (!split) {
        for (int k = 0; k < 4; k++) p.fmaps[1][k] = p.fmaps[0][k];
        for (int k = 0; k < 6; k++) p.bmaps[1][k] = p.bmaps[0][k];
    }
    if (!ok) return false;
    ok = cudaFuncSetAttribute(k_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F_SMEM) == cudaSuccess &&
         cudaFuncSetAttribute(k_forward_tc_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F_SMEM) ==
             cudaSuccess &&
         cudaFuncSetAttribute(k_backproject_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B_SMEM) ==
             cudaSuccess &&
         cudaFuncSetAttribute(k_backproject_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B_SMEM) ==
             cudaSuccess;
    p.ready = ok;
    return ok;
}

// ---------------------------------------------------------------- autotuning

namespace {
std::mutex g_tune_mu;
struct TuneChoice {
    int kper = 1;
    bool fused = false;
    float ms[4] = {0.f, 0.f, 0.f, 0.f};
};
std::map<std::tuple<int, int, int, bool>, TuneChoice> g_tune;   // (device, N, X, split) -> choice
int g_tune_mode = 1;
}  // namespace

int set_autotune(int mode)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    int old = g_tune_mode;
    if (mode == 0 || mode == 1 || mode == 2) g_tune_mode = mode;
    return old;
}

static void apply_kper(TcPlanes &p, int kper)
{
    const int nk = p.Xpad / BK;
    p.fwd_kper = kper;
    p.fwd_splits = (nk + kper - 1) / kper;
}

bool tc_autotune(TcPlanes &p, float2 *part, TabEntry *tab, float2 *v, cudaStream_t s)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, p.N, p.X, p.split);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (g_tune_mode == 0) return true;                      // heuristic split
        if (g_tune_mode == 2) {                                 // heuristic split, fused forward
            p.fwd_fused = !p.split;
            return true;
        }
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            apply_kper(p, it->second.kper);
            p.fwd_fused = it->second.fused;
            for (int k = 0; k < 4; k++) p.tune_ms[k] = it->second.ms[k];
            return true;
        }
    }
    const int nk = p.Xpad / BK, T = p.Npad / BM, pairs = T * (T + 1) / 2;
    const int base = p.fwd_splits;
    std::vector<int> kpers;
    for (int m : {1, 2, 3, 4, -2}) {                             // -2: half the split
        int sp = m > 0 ? base * m : std::max(1, base / 2);
        sp = std::min(sp, p.fwd_max_splits);
        const int kper = (nk + sp - 1) / sp;
        if (std::find(kpers.begin(), kpers.end(), kper) == kpers.end()) kpers.push_back(kper);
    }
    Maps4 hi{p.fmaps[0][0], p.fmaps[0][1], p.fmaps[0][2], p.fmaps[0][3]};
    Maps4 lo{p.fmaps[1][0], p.fmaps[1][1], p.fmaps[1][2], p.fmaps[1][3]};
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return false;
    int best = p.fwd_kper;
    float best_ms = 1e30f;
    bool ok = true;
    for (int kper : kpers) {
        const int sp = (nk + kper - 1) / kper;
        float tot = 0.f;
        for (int rep = 0; rep < 3 && ok; rep++) {              // first launch warms up
            ok = cudaEventRecord(a, s) == cudaSuccess;
            k_forward_tc<<<dim3(pairs, sp), 192, F_SMEM, s>>>(hi, lo, p.split ? 3 : 1, p.N, T, nk, kper, part, p.err);
            ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(b, s) == cudaSuccess &&
                 cudaEventSynchronize(b) == cudaSuccess;
            float ms = 0.f;
            ok = ok && cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
            if (rep > 0) tot += ms;
        }
        if (!ok) break;
        if (tot < best_ms) {
            best_ms = tot;
            best = kper;
        }
        p.tuned++;
    }
    TuneChoice ch;
    ch.kper = best;
    apply_kper(p, best);
    // plain BF16: the separate synthesis pass (both operand sets, as an update runs it) plus the
    // forward GEMM, against the back-projection's synthesis alone plus the fused forward, on
    // tables holding covered entries (every entry then costs its full synthesis)
    if (ok && !p.split && tab && v) {
        ok = cudaMemsetAsync(tab, 0, sizeof(TabEntry) * (size_t)p.N * p.X, s) == cudaSuccess &&
             cudaMemsetAsync(v, 0, sizeof(float2) * (size_t)p.X, s) == cudaSuccess;
        const double f = 5e5, c0 = 1500.0;
        auto timed = [&](auto &&launch) {
            float tot = 0.f;
            for (int rep = 0; rep < 3 && ok; rep++) {
                ok = cudaEventRecord(a, s) == cudaSuccess;
                launch();
                ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(b, s) == cudaSuccess &&
                     cudaEventSynchronize(b) == cudaSuccess;
                float ms = 0.f;
                ok = ok && cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
                if (rep > 0) tot += ms * 0.5f;
            }
            return tot;
        };
        ch.ms[0] = timed([&] { launch_synth_both_tc(p, tab, v, f, c0, s); });
        ch.ms[1] = timed([&] { launch_forward_tc(p, part, s); });
        ch.ms[2] = timed([&] { launch_synth_bp_tc(p, tab, f, c0, s); });
        // the fused form once; timed again only if it is not already twice the separate pass
        float once = 0.f;
        if (ok) {
            ok = cudaEventRecord(a, s) == cudaSuccess;
            launch_forward_tc_fused(p, tab, v, f, c0, part, s);
            ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(b, s) == cudaSuccess &&
                 cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&once, a, b) == cudaSuccess;
        }
        ch.ms[3] = once;
        if (ok && once < 2.f * (ch.ms[0] + ch.ms[1]))
            ch.ms[3] = timed([&] { launch_forward_tc_fused(p, tab, v, f, c0, part, s); });
        ch.fused = ok && ch.ms[2] + ch.ms[3] < ch.ms[0] + ch.ms[1];
        p.tuned += 2;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!ok) return false;
    unsigned zero = 0;
    if (cudaMemcpyAsync(p.err, &zero, sizeof zero, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return false;
    p.fwd_fused = ch.fused;
    for (int k = 0; k < 4; k++) p.tune_ms[k] = ch.ms[k];
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.emplace(key, ch);
    return true;
}

void tc_free(TcPlanes &p, cudaStream_t st)
{
    void *ps[] = {p.fplanes, p.bplanes, p.rsplanes, p.bpart, p.err};
    for (void *q : ps)
        if (q) cudaFreeAsync(q, st);
    p = TcPlanes{};
}

static float green_const_tc(double f, double c0)
{
    return (float)(1.0 / sqrt(8.0 * 3.14159265358979323846 * (2.0 * 3.14159265358979323846 * f) / c0));
}

void launch_synth_fwd_tc(TcPlanes &p, const TabEntry *tab, const float2 *v, double f, double c0, cudaStream_t s)
{
    size_t n = (size_t)p.N * p.X;
    float fhi = (float)f, flo = (float)(f - (double)fhi);
    k_synth_fwd_tc<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tab, v, p.N, p.X, p.Xpad, p.fwd_pstride, fhi, flo,
                                                               green_const_tc(f, c0),
                                                               static_cast<__nv_bfloat16 *>(p.fplanes), p.split);
}

int launch_forward_tc_fused(TcPlanes &p, const TabEntry *tab, const float2 *v, double f, double c0, float2 *part,
                            cudaStream_t s)
{
    const int T = p.Npad / BM, pairs = T * (T + 1) / 2;
    const float fhi = (float)f, flo = (float)(f - (double)fhi);
    k_forward_tc_fused<<<dim3(pairs, p.fwd_splits), 192, F_SMEM, s>>>(tab, v, p.N, p.X, T, p.Xpad / BK, p.fwd_kper,
                                                                      fhi, flo, green_const_tc(f, c0), part, p.err);
    return p.fwd_splits;
}

int launch_forward_tc(TcPlanes &p, float2 *part, cudaStream_t s)
{
    int T = p.Npad / BM, pairs = T * (T + 1) / 2;
    Maps4 hi{p.fmaps[0][0], p.fmaps[0][1], p.fmaps[0][2], p.fmaps[0][3]};
    Maps4 lo{p.fmaps[1][0], p.fmaps[1][1], p.fmaps[1][2], p.fmaps[1][3]};
    k_forward_tc<<<dim3(pairs, p.fwd_splits), 192, F_SMEM, s>>>(hi, lo, p.split ? 3 : 1, p.N, T, p.Xpad / BK,
                                                                p.fwd_kper, part, p.err);
    return p.fwd_splits;
}

// Shared memory and persistent grid of k_synth_tc<FWD, SPLIT> (set up once per instance).
template <bool FWD, bool SPLIT>
static int synth_grid(size_t &smem)
{
    smem = 2 * kSynSlots * sizeof(TabEntry) + (SPLIT ? 12 : 6) * 32 * 34 * sizeof(__nv_bfloat16);
    static int blocks = 0;
    if (blocks == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_synth_tc<FWD, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_synth_tc<FWD, SPLIT>, 256, smem);
        blocks = sms * (per_sm > 0 ? per_sm : 1);
    }
    return blocks;
}

template <bool FWD, bool SPLIT>
static void synth_launch(TcPlanes &p, const TabEntry *tab, const float2 *v, double f, double c0, cudaStream_t s)
{
    const float fhi = (float)f, flo = (float)(f - (double)fhi);
    const int XT = (p.X + 31) / 32, ntiles = XT * ((p.N + 31) / 32);
    size_t smem = 0;
    int grd = synth_grid<FWD, SPLIT>(smem);
    if (grd > ntiles) grd = ntiles;
    k_synth_tc<FWD, SPLIT><<<grd, 256, smem, s>>>(tab, p.N, p.X, p.Npad, p.bp_pstride, fhi, flo, green_const_tc(f, c0),
                                                  static_cast<__nv_bfloat16 *>(p.bplanes), v, FWD ? p.Xpad : 0,
                                                  FWD ? p.fwd_pstride : 0,
                                                  FWD ? static_cast<__nv_bfloat16 *>(p.fplanes) : nullptr, XT, ntiles);
}

void launch_synth_bp_tc(TcPlanes &p, const TabEntry *tab, double f, double c0, cudaStream_t s)
{
    if (p.split)
        synth_launch<false, true>(p, tab, nullptr, f, c0, s);
    else
        synth_launch<false, false>(p, tab, nullptr, f, c0, s);
}

void launch_synth_both_tc(TcPlanes &p, const TabEntry *tab, const float2 *v, double f, double c0, cudaStream_t s)
{
    if (p.split)
        synth_launch<true, true>(p, tab, v, f, c0, s);
    else
        synth_launch<true, false>(p, tab, v, f, c0, s);
}

// One thread waits, with the bound every tensor-core kernel uses, on an mbarrier that nothing
// signals: flag = 1 when the wait gave up.
__global__ void k_wait_selftest(unsigned *flag)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        *flag = mbar_wait(&bar, 0) ? 0u : 1u;
    }
}

void launch_wait_selftest(unsigned *flag, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(flag);
}

void launch_backproject_tc(TcPlanes &p, const float2 *Rs, int weight_mode, float2 *gpart, cudaStream_t s)
{
    size_t nn = (size_t)p.N * p.N;
    k_rs_planes<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(Rs, p.N, p.Npad,
                                                             static_cast<__nv_bfloat16 *>(p.rsplanes), p.split);
    dim3 grd(p.Npad / BN, p.Xp / BM);
    Maps6 hi{p.bmaps[0][0], p.bmaps[0][1], p.bmaps[0][2], p.bmaps[0][3], p.bmaps[0][4], p.bmaps[0][5]};
    Maps6 lo{p.bmaps[1][0], p.bmaps[1][1], p.bmaps[1][2], p.bmaps[1][3], p.bmaps[1][4], p.bmaps[1][5]};
    const __nv_bfloat16 *bp = static_cast<const __nv_bfloat16 *>(p.bplanes);
    const float sgn = weight_mode == 0 ? -1.f : 1.f;
    if (p.split)
        k_backproject_tc<true><<<grd, 192, B_SMEM, s>>>(hi, lo, bp, p.bp_pstride, p.Npad, p.Npad / BK, sgn, p.bpart,
                                                        p.Xp, p.err);
    else
        k_backproject_tc<false><<<grd, 192, B_SMEM, s>>>(hi, lo, bp, p.bp_pstride, p.Npad, p.Npad / BK, sgn, p.bpart,
                                                         p.Xp, p.err);
    k_bp_reduce<<<(p.X + 255) / 256, 256, 0, s>>>(p.bpart, p.Npad / BN, p.Xp, p.X, gpart);
}

}  // namespace rbx
