// Internal declarations of the rbx CUDA library (not part of the public ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include "../../include/rbx.h"

namespace rbx {

// Field map: 8 floats per node in three planes, so a lossless, smoothed trace touches only
// the first two (24 B per node): [nxy] float4 (n, n_x, n_y, n_xx), [nxy] float2 (n_xy, n_yy),
// [nxy] float2 (alpha, n_raw).
constexpr int kFieldStride = 8;
constexpr uint32_t kUncovered = 0xFFFFFFFFu;
constexpr int kMaxSteps = 2047;          // ray samples index i < 2048 (11 bits of the key)
constexpr int kMaxXducers = 4095;        // ray index j < 4096 (12 bits of the key)
constexpr int kHistSlots = 64;           // device history of per-update scalars (one slot per update)
constexpr int kHistStride = 12;          // doubles per slot: |R|^2, sum dc^2, max|dc|, sum dm^2, counters[0..5], tc err

// One (transducer, mask node) table entry, 16 bytes. The first 8 bytes, read as a
// little-endian u64, are the ordering key (T bits, triangle id, K): the rasteriser keeps
// the smallest key per node with a 128-bit compare-and-swap.
struct __align__(16) TabEntry {
    uint32_t idk;   // (triangle id << 8) | K ; kUncovered when no triangle covered the node
    float T;        // travel time [s]
    float a;        // reduced amplitude [m^-1/2]
    float gam;      // ray direction angle [rad]
};

struct RayParams {
    int N, X, nx, ny;
    float dx, x0, y0, R, ds, inv_dx, rmask;
    int maxs;
    const double *beta;   // [N] position angles of the transducers (device); nullptr: uniform ring 2 pi e / N
};

// 1/v for v finite and away from 0 and the denormal range (a slowness, a triangle's edge
// sum, an amplitude times a constant): the hardware approximation refined by one
// Newton-Raphson step, r <- r + r (1 - v r).
__device__ __forceinline__ float rcp_nr(float v)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return fmaf(fmaf(-v, r, 1.f), r, r);
}

// Angular density (step a4): |d gamma / d e| Delta e as half the difference of the direction
// angles of the two neighbouring transducers, wrapped to [-pi, pi). One expression for every
// kernel that forms it, so they agree bit for bit.
__device__ __forceinline__ float dgamma_of(float gam_next, float gam_prev)
{
    const float PI = 3.14159265358979f, TWO_PI = 6.28318530717959f, INV_TWO_PI = 0.159154943091895f;
    float d = gam_next - gam_prev;
    d = d - TWO_PI * floorf((d + PI) * INV_TWO_PI);
    return 0.5f * fabsf(d);
}

// BF16 tensor-core operands of one job: planar complex planes, their TMA descriptors and
// the back-projection partials (k_gemm_tc.cu).
struct TcPlanes {
    int N = 0, X = 0, Npad = 0, Xpad = 0, Xp = 0, sms = 0;
    size_t fwd_pstride = 0, bp_pstride = 0;
    int fwd_splits = 1, fwd_kper = 1;
    int fwd_max_splits = 1;    // largest K split the autotuner may pick (sizes the partials)
    int tuned = 0;             // candidates timed for this job (0: heuristic or cached choice)
    bool fwd_fused = false;    // the forward forms its operands from the tables (k_forward_tc_fused)
    float tune_ms[4] = {0.f, 0.f, 0.f, 0.f};   // tuner's times: both synthesis passes, forward GEMM,
                                               // back-projection synthesis alone, fused forward
    bool split = false;        // split BF16: every plane set is followed by its lo set
    void *fplanes = nullptr;   // [4][Npad][Xpad] bf16: Gre, Gim, (Gv)re, (Gv)im
    void *bplanes = nullptr;   // [6][Xp][Npad] bf16: u, conj(kappa) u, kappa u (re, im)
    void *rsplanes = nullptr;  // [2][Npad][Npad] bf16: R_s re, im
    float2 *bpart = nullptr;   // [Npad/128][Xp] partial back-projection
    unsigned *err = nullptr;   // bounded-wait timeouts of the tensor-core kernels
    CUtensorMap fmaps[2][4], bmaps[2][6];   // [hi, lo]
    bool ready = false;
};

// Device workspace of one job.
struct Workspace {
    int N = 0, X = 0, nx = 0, ny = 0;
    int *node2x = nullptr, *idx = nullptr;
    int4 *rows = nullptr;       // per grid row: (compact index of first mask node, first ix, last ix)
    float *c = nullptr, *ns = nullptr, *tmp = nullptr, *fields = nullptr;
    double *ns64 = nullptr, *tmp64 = nullptr;
    TabEntry *tab = nullptr;
    float *dg = nullptr;
    float4 *exits = nullptr;
    float2 *G = nullptr, *U = nullptr, *kap = nullptr;
    float2 *v = nullptr;        // Born weight Upsilon_m dA (m - m_s) per mask node (complex when lossy)
    float *alpha0 = nullptr;    // absorption map alpha0 [ny][nx], Np (rad/s)^-y m^-1 (lossy jobs only)
    double *as64 = nullptr;     // smoothed alpha0 (lossy jobs only)
    double *dmacc = nullptr;    // sum of a frequency set's search directions per mask node
    float4 *linked = nullptr;   // linked rays of the direct term [N][N] (0, T, a, K)
    double *beta = nullptr;     // [N] position angles of caller-placed transducers; nullptr: uniform ring
    float2 *gdir = nullptr, *D = nullptr, *R = nullptr, *Rs = nullptr, *part = nullptr, *gpart = nullptr;
    float2 *data = nullptr;
    double *red = nullptr;           // reduction scratch
    double *hist = nullptr;          // [kHistSlots][kHistStride] per-update scalars
    unsigned long long *counters = nullptr;   // [0] covered entries [1] clamped [2] bad rays [3] CAS bound [4] m <= 0 [5] bad model [6] mask count [7] uniform radius (float bits)
    int fwd_splits = 1;
    TcPlanes tc;
};

// ---------------------------------------------------------------- kernels (launchers)
// k_fields.cu
void launch_mask(const rbx_geometry &g, int *node2x, int *count, cudaStream_t s);
void launch_mask_idx(const int *node2x, int nxy, int *idx, cudaStream_t s);
// Absorption of a lossy job (Szabo power law): alpha = alpha0 omega^y, rays on
// 1/c + alpha0 tan(pi y/2) omega^(y-1). alpha0 == nullptr: lossless.
struct Lossy {
    const float *alpha0 = nullptr;
    double *as64 = nullptr;
    double y = 0.0;
};
void launch_smooth_fields(const rbx_geometry &g, const float *c, int w, double *tmp64, double *ns64, float *ns,
                          float *fields, const Lossy &ab, double f, bool raw, cudaStream_t s);
void launch_check_model(const float *c, int n, unsigned long long *flag, cudaStream_t s);
void launch_check_alpha(const float *a, int n, unsigned long long *flag, cudaStream_t s);
void launch_fill(float *p, float v, size_t n, cudaStream_t s);

// k_rays.cu
void launch_uniform_radius(const float *fields, const RayParams &p, unsigned long long *ru, cudaStream_t s);
void launch_trace_raster(const float *fields, const int4 *rows, TabEntry *tab, float4 *exits, const RayParams &p,
                         unsigned long long *counters, bool lossy, bool raw, cudaStream_t s);
// One job of a persistent grouped trace (the batched form): its buffers and ray parameters,
// and the range of work items it owns, [item0, item0 + nwarps * ceil(N / 4)).
struct TraceJob {
    const float *F;
    const int4 *rows;
    TabEntry *tab;
    float4 *exits;
    unsigned long long *counters;
    RayParams p;
    int item0, nwarps;
};
// Up to kMaxGroup jobs of one grouped trace launch, item0 ascending from 0; total = all items.
constexpr int kMaxGroup = 64;
struct TraceGroup {
    int njobs, total;
    TraceJob j[kMaxGroup];
};
// Work items of a job in the grouped trace (the per-job kernel's blocks).
int trace_items(int N, int *nwarps);
// Resident blocks of the grouped trace on this device (its grid).
int trace_grouped_blocks(bool lossy, bool raw, int max_ny);
// The traces of g's jobs as one persistent launch of `blocks` blocks taking items from *next
// (zeroed by the caller).
void launch_trace_grouped(const TraceGroup &g, int max_ny, int blocks, int *next, bool lossy, bool raw, cudaStream_t s);
void launch_mask_rows(const int *node2x, int nx, int ny, int4 *rows, cudaStream_t s);
// secant-linked rays of the direct term, linked[e][r] = (0, T, a, K) (maxit new rays per pair at
// most), and the direct Green's function of one frequency from them
void launch_link_rays(const float *fields, const RayParams &p, const float4 *exits, int maxit, float4 *linked,
                      unsigned long long *counters, bool lossy, bool raw, cudaStream_t s);
void launch_green_linked(const float4 *linked, int N, double f, double c0, float2 *g, cudaStream_t s);
void launch_dgamma(const TabEntry *tab, float *dg, int N, int X, cudaStream_t s);
void launch_direct_green(const float4 *exits, int N, const double *beta, double f, double c0, float2 *g,
                         unsigned long long *counters,
                         cudaStream_t s);
void launch_set_tables(const float *T, const float *a, const float *gam, const uint8_t *K, TabEntry *tab, size_t n,
                       unsigned long long *counters, cudaStream_t s);
void launch_get_tables(const TabEntry *tab, float *T, float *a, float *gam, uint8_t *K, size_t n, cudaStream_t s);

// k_gemm_simt.cu
void launch_synth_fwd(const TabEntry *tab, int N, int X, double f, double c0, float2 *G, cudaStream_t s);
void launch_synth_bp(const TabEntry *tab, const float *dg, int N, int X, double f, double c0, float2 *U,
                     float2 *kap, cudaStream_t s);
// Born weights v[x] = Upsilon_m dA (m - m_s) (rough part) or Upsilon_m dA dm[x], with
// Upsilon_m = omega c k~ at the node (omega^2 when lossless; c = current model).
void launch_born_weights_rough(const float *c, const double *ns64, const int *idx, int X, double f, double dA,
                               const Lossy &ab, float2 *v, cudaStream_t s);
void launch_born_weights_dm(const float *dm, const float *c, const int *idx, int X, double f, double dA,
                            const Lossy &ab, float2 *v, cudaStream_t s);
int forward_splits(int N, int X);
void launch_forward_simt(const float2 *G, const float2 *v, int N, int X, int splits, float2 *part, cudaStream_t s);
void launch_forward_reduce(const float2 *part, int N, int splits, float2 *D, cudaStream_t s);
// mode 0: preconditioned (A = U, conj(kap) U; W = U, kap U); mode 1: plain adjoint (A = W = conj(G))
void launch_backproject_simt(const float2 *A, const float2 *kap, const float2 *Rs, int N, int X, int mode,
                             float2 *gpart, cudaStream_t s);

// k_gemm_tc.cu (BF16 tensor cores)
bool tc_setup(TcPlanes &p, int N, int X, bool split, cudaStream_t s);
// Choose the forward K split by timing the candidates on this job's planes (once per shape
// and process; later jobs of the shape reuse the choice). part holds fwd_max_splits partials.
bool tc_autotune(TcPlanes &p, float2 *part, TabEntry *tab, float2 *v, cudaStream_t s);
int set_autotune(int mode);
void tc_free(TcPlanes &p, cudaStream_t s);
void launch_synth_fwd_tc(TcPlanes &p, const TabEntry *tab, const float2 *v, double f, double c0, cudaStream_t s);
int launch_forward_tc(TcPlanes &p, float2 *part, cudaStream_t s);
// The forward with its operands formed from the tables in the contraction (no planes).
int launch_forward_tc_fused(TcPlanes &p, const TabEntry *tab, const float2 *v, double f, double c0, float2 *part,
                            cudaStream_t s);
void launch_synth_bp_tc(TcPlanes &p, const TabEntry *tab, double f, double c0, cudaStream_t s);
// a bounded wait on a barrier nothing signals (flag = 1 when it gave up)
void launch_wait_selftest(unsigned *flag, cudaStream_t s);
// both operand sets of an update in one pass over the tables (forward planes with weights v)
void launch_synth_both_tc(TcPlanes &p, const TabEntry *tab, const float2 *v, double f, double c0, cudaStream_t s);
void launch_backproject_tc(TcPlanes &p, const float2 *Rs, int weight_mode, float2 *gpart, cudaStream_t s);

// k_update.cu
void launch_residual(const float2 *gdir, const float2 *D, const float2 *data, int N, float2 *R, float2 *Rs,
                     double *red, cudaStream_t s);
void launch_symmetrize(const float2 *R, int N, float2 *Rs, cudaStream_t s);
void launch_combine_adjoint(const float2 *gpart, int X, int mode, int weight_mode, double scale, float2 *out,
                            cudaStream_t s);
// plain adjoint of a lossy job: out[x] = dA conj(Upsilon_m[x]) gpart[x]
void launch_combine_adjoint_lossy(const float2 *gpart, const float *c, const int *idx, int X, double f, double dA,
                                  const Lossy &ab, float2 *out, cudaStream_t s);
void launch_acc_scalar(const double *src, double *dst, bool first, cudaStream_t s);
void launch_update(const float2 *gpart, const int *node2x, int nx, int ny, int X, int weight_mode, double f,
                   double df, double tau, double c0, float *c, double *red, unsigned long long *counters,
                   const Lossy &ab, double *acc, int mode, cudaStream_t s);
void launch_snapshot(const double *r2, const double *upd3, const unsigned long long *counters, const unsigned *tc_err,
                     unsigned long long n_entries, double *slot, cudaStream_t s);
int residual_blocks(int N);
int update_blocks(int nx, int ny);

// rbx_api.cu: hooks for the server (C++ linkage, not part of the C ABI)
rbx_status job_enqueue_sweep(rbx_job *j, const double *freqs, int nf, const void *data_dev);
rbx_status job_read_sweep(rbx_job *j, int nf, rbx_stats *last);
cudaStream_t job_stream(const rbx_job *j);
float *job_model(rbx_job *j);
size_t job_bytes_estimate(const rbx_geometry &g, int nf);

}  // namespace rbx
