// C ABI of the rbx library: job state, argument checks and the order of the steps of one
// Hessian-free update (declared in include/rbx.h).
#include "rbx_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace rbx;

namespace rbx {
void launch_add_offdiag(const float2 *a, const float2 *b, int N, float2 *out, cudaStream_t s);
}

enum { EV_START, EV_FIELDS, EV_TRACE, EV_TABLES, EV_GDIR, EV_SYNTH_F, EV_GEMM_F, EV_RESID, EV_SYNTH_B, EV_GEMM_B,
       EV_UPDATE, EV_COUNT };

struct rbx_job {
    cudaStream_t stream = nullptr;
    rbx_geometry g{};
    bool has_geom = false, has_tables = false, ns_valid = false;
    int ns_window = 0;
    double ns_freq = 0.0;      // frequency the fields were made for (lossy fields depend on it)
    bool lossy = false;        // absorption map set (rbx_set_absorption)
    bool raw = false;          // integration on the non-smoothed map (rbx_set_integration)
    int link_iters = 0;        // secant ray linking of the direct term, new rays per pair (0: off)
    bool linked_valid = false; // w.linked holds the linked rays of the current tables
    bool dg_valid = false;     // w.dg holds the angular density of the current tables
    double abs_y = 0.0;
    Workspace w;
    int *d_count = nullptr;
    std::string err;
    cudaEvent_t ev[EV_COUNT]{};
    cudaEvent_t *evp = nullptr;         // the event set record() writes: ev, or a slot's set
    cudaEvent_t *slot_ev = nullptr;     // [kHistSlots][EV_COUNT] (rbx_set_slot_timing)
    long long slot_launches[kHistSlots] = {};
    long long slot_l0 = 0;     // launch count when the update being queued began
    // rbx_update_frequency_host: a copy stream for the data, which the trace does not read
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_in_free = nullptr, ev_in_ready = nullptr;
    long long launches = 0;
};

static rbx_status fail(rbx_job *j, rbx_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (j) j->err = buf;
    return st;
}

#define CUDA_TRY(job, call)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(job, RBX_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
    } while (0)
#define LAUNCHED(job, n)                                                                     \
    do {                                                                                     \
        (job)->launches += (n);                                                              \
        CUDA_TRY(job, cudaGetLastError());                                                   \
    } while (0)
#define NEED(job, cond, st, msg)                                                             \
    do {                                                                                     \
        if (!(cond)) return fail(job, st, "%s", msg);                                        \
    } while (0)

// Job workspaces come from the device's stream-ordered pool: allocating and releasing them
// never waits for other jobs' work (a plain cudaFree would synchronise the whole device).
// The pool keeps released memory for reuse (release threshold raised once per device).
static void keep_pool_memory()
{
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    done[dev] = true;
}

template <class T>
static cudaError_t dalloc(T *&p, size_t n, cudaStream_t s)
{
    return cudaMallocAsync(reinterpret_cast<void **>(&p), (n ? n : 1) * sizeof(T), s);
}

static void free_ws(Workspace &w, cudaStream_t s)
{
    void *ps[] = {w.hist, w.node2x, w.idx, w.rows, w.c, w.ns, w.tmp, w.fields, w.ns64, w.tmp64, w.tab, w.dg, w.exits, w.G, w.U,
                  w.kap, w.v, w.gdir, w.D, w.R, w.Rs, w.part, w.gpart, w.data, w.red, w.counters, w.alpha0, w.as64,
                  w.dmacc, w.linked, w.beta};
    for (void *p : ps)
        if (p) cudaFreeAsync(p, s);
    tc_free(w.tc, s);
    w = Workspace{};
}

// Odd smoothing window in grid points: 13, 11, 9, 7 on a 1 mm grid below 0.4, 0.7, 1 MHz
// and above; scaled by (1 mm / dx) to the nearest odd integer (Sec. 6.2, Sec. 6.3.2).
static int window_for(double f, double dx)
{
    double w1 = f < 0.4e6 ? 13.0 : (f < 0.7e6 ? 11.0 : (f < 1.0e6 ? 9.0 : 7.0));
    double w = w1 * (1e-3 / dx);
    int k = (int)std::floor((w - 1.0) / 2.0 + 0.5);
    if (k < 0) k = 0;
    return 2 * k + 1;
}

static int max_steps(const rbx_geometry &g) { return (int)std::ceil(3.0 * g.ring_radius / g.ds) + 8; }

static float elapsed(const rbx_job *j, int a, int b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, j->evp[a], j->evp[b]) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

static rbx_status record(rbx_job *j, int k)
{
    CUDA_TRY(j, cudaEventRecord(j->evp[k], j->stream));
    return RBX_OK;
}

extern "C" {

rbx_status rbx_create(rbx_job **out, void *cuda_stream)
{
    if (!out) return RBX_EINVAL;
    *out = nullptr;
    rbx_job *j = new (std::nothrow) rbx_job();
    if (!j) return RBX_ENOMEM;
    j->stream = static_cast<cudaStream_t>(cuda_stream);   // NULL: the legacy default stream
    j->evp = j->ev;
    for (int k = 0; k < EV_COUNT; k++) {
        if (cudaEventCreate(&j->ev[k]) != cudaSuccess) {
            rbx_destroy(j);
            return RBX_ECUDA;
        }
    }
    *out = j;
    return RBX_OK;
}

rbx_status rbx_destroy(rbx_job *j)
{
    if (!j) return RBX_EINVAL;
    cudaStreamSynchronize(j->stream);
    free_ws(j->w, j->stream);
    if (j->d_count) cudaFreeAsync(j->d_count, j->stream);
    cudaStreamSynchronize(j->stream);
    for (int k = 0; k < EV_COUNT; k++)
        if (j->ev[k]) cudaEventDestroy(j->ev[k]);
    if (j->copy_stream) {
        cudaStreamSynchronize(j->copy_stream);
        cudaStreamDestroy(j->copy_stream);
    }
    if (j->ev_in_free) cudaEventDestroy(j->ev_in_free);
    if (j->ev_in_ready) cudaEventDestroy(j->ev_in_ready);
    if (j->slot_ev) {
        for (int k = 0; k < kHistSlots * EV_COUNT; k++)
            if (j->slot_ev[k]) cudaEventDestroy(j->slot_ev[k]);
        delete[] j->slot_ev;
    }
    delete j;
    return RBX_OK;
}

const char *rbx_last_error(const rbx_job *j) { return j ? j->err.c_str() : "null job"; }

rbx_status rbx_synchronize(rbx_job *j)
{
    if (!j) return RBX_EINVAL;
    CUDA_TRY(j, cudaStreamSynchronize(j->stream));
    return RBX_OK;
}

rbx_status rbx_set_geometry(rbx_job *j, const rbx_geometry *geom, const double *xducer_xy)
{
    if (!j || !geom) return RBX_EINVAL;
    const rbx_geometry &g = *geom;
    NEED(j, g.nx >= 4 && g.ny >= 4 && std::isfinite(g.dx) && g.dx > 0, RBX_EINVAL, "grid must be >= 4x4 with dx > 0");
    NEED(j, g.n_xducers >= 3 && g.n_xducers <= kMaxXducers, RBX_EINVAL, "n_xducers must be in [3, 4095]");
    NEED(j, std::isfinite(g.ring_radius) && g.ring_radius > 0, RBX_EINVAL, "ring_radius must be > 0");
    NEED(j, g.mask_radius > 0 && g.mask_radius <= g.ring_radius, RBX_EINVAL, "mask_radius must be in (0, R]");
    NEED(j, std::isfinite(g.c0) && g.c0 > 0, RBX_EINVAL, "c0 must be > 0");
    NEED(j, std::isfinite(g.ds) && g.ds > 0, RBX_EINVAL, "ds must be > 0");
    NEED(j, g.weight_mode == 0 || g.weight_mode == 1, RBX_EINVAL, "weight_mode must be 0 or 1");
    NEED(j, std::isfinite(g.tau), RBX_EINVAL, "tau must be finite");
    NEED(j, g.precision >= RBX_FP32 && g.precision <= RBX_BF16X3, RBX_EINVAL,
         "precision must be RBX_FP32, RBX_BF16 or RBX_BF16X3");
    double xl = g.x0, xr = g.x0 + (g.nx - 1) * g.dx, yl = g.y0, yr = g.y0 + (g.ny - 1) * g.dx;
    NEED(j, xl <= -g.ring_radius - g.dx && xr >= g.ring_radius + g.dx && yl <= -g.ring_radius - g.dx &&
                yr >= g.ring_radius + g.dx,
         RBX_EINVAL, "the grid must contain the ring with one node to spare");
    NEED(j, max_steps(g) <= kMaxSteps, RBX_EINVAL, "ring_radius / ds too large (rays limited to 2047 steps)");
    NEED(j, (double)g.nx * g.ny < 2e9, RBX_EINVAL, "grid too large");
    // caller-placed transducers (Sec. 2.1): on the ring, counterclockwise, once around
    std::vector<double> beta;
    if (xducer_xy) {
        const double TWO_PI = 6.283185307179586476925;
        beta.resize(g.n_xducers);
        for (int e = 0; e < g.n_xducers; e++) {
            const double x = xducer_xy[2 * e], y = xducer_xy[2 * e + 1];
            NEED(j, std::isfinite(x) && std::isfinite(y) && std::fabs(std::hypot(x, y) - g.ring_radius) <= 1e-6 * g.ring_radius,
                 RBX_EINVAL, "transducer positions must lie on the ring (|x_e| = ring_radius within 1e-6 relative)");
            beta[e] = std::atan2(y, x);
        }
        double turn = 0.0;
        for (int e = 0; e < g.n_xducers; e++) {
            double d = beta[(e + 1) % g.n_xducers] - beta[e];
            d -= TWO_PI * std::floor(d / TWO_PI);
            NEED(j, d > 0.0, RBX_EINVAL, "transducer positions must be distinct");
            turn += d;
        }
        NEED(j, std::fabs(turn - TWO_PI) <= 1e-9, RBX_EINVAL,
             "transducer positions must run counterclockwise around the ring once, in index order");
    }

    CUDA_TRY(j, cudaStreamSynchronize(j->stream));
    free_ws(j->w, j->stream);
    keep_pool_memory();
    j->has_geom = j->has_tables = j->ns_valid = j->lossy = j->raw = false;
    j->link_iters = 0;
    Workspace &w = j->w;
    w.N = g.n_xducers;
    w.nx = g.nx;
    w.ny = g.ny;
    const size_t nxy = (size_t)g.nx * g.ny, N = w.N;
    if (!j->d_count) CUDA_TRY(j, dalloc(j->d_count, 1, j->stream));
#define ALLOC(p, n)                                                                                   \
    do {                                                                                              \
        if (dalloc(p, n, j->stream) != cudaSuccess) {                                                 \
            cudaGetLastError();                                                                       \
            free_ws(w, j->stream);                                                                    \
            return fail(j, RBX_ENOMEM, "device allocation of %s (%zu elements) failed", #p, (size_t)(n)); \
        }                                                                                             \
    } while (0)
    ALLOC(w.node2x, nxy);
    launch_mask(g, w.node2x, j->d_count, j->stream);
    LAUNCHED(j, 1);
    int X = 0;
    CUDA_TRY(j, cudaMemcpyAsync(&X, j->d_count, sizeof(int), cudaMemcpyDeviceToHost, j->stream));
    CUDA_TRY(j, cudaStreamSynchronize(j->stream));
    NEED(j, X > 0, RBX_EINVAL, "the mask contains no grid node");
    w.X = X;
    w.fwd_splits = forward_splits(w.N, X);
    const size_t NX = N * (size_t)X;
    ALLOC(w.idx, X);
    ALLOC(w.rows, (size_t)g.ny);
    ALLOC(w.c, nxy);
    ALLOC(w.ns, nxy);
    ALLOC(w.ns64, nxy);
    ALLOC(w.tmp64, nxy);
    ALLOC(w.fields, nxy * kFieldStride);
    ALLOC(w.tab, NX);
    ALLOC(w.dg, NX);
    ALLOC(w.exits, N * (N - 1));
    ALLOC(w.G, NX);
    if (g.precision == RBX_FP32) {   // FP32 back-projection operands (the tensor-core path has its own)
        ALLOC(w.U, NX);
        ALLOC(w.kap, NX);
    }
    ALLOC(w.v, X);
    ALLOC(w.gdir, N * N);
    ALLOC(w.D, N * N);
    ALLOC(w.R, N * N);
    ALLOC(w.Rs, N * N);
    ALLOC(w.data, N * N);
    if (g.precision != RBX_FP32) {
        if (!tc_setup(w.tc, w.N, X, g.precision == RBX_BF16X3, j->stream)) {
            cudaGetLastError();
            free_ws(w, j->stream);
            return fail(j, RBX_ENOMEM, "tensor-core operand set-up failed (allocation or TMA descriptor)");
        }
        if (w.tc.fwd_max_splits > w.fwd_splits) w.fwd_splits = w.tc.fwd_max_splits;
    }
    ALLOC(w.part, (size_t)w.fwd_splits * N * N);
    if (g.precision != RBX_FP32 && !tc_autotune(w.tc, w.part, w.tab, w.v, j->stream)) {
        cudaGetLastError();
        free_ws(w, j->stream);
        return fail(j, RBX_ECUDA, "autotuning of the tensor-core forward failed");
    }
    ALLOC(w.gpart, 2 * (size_t)X);
    // residual partials + total, then the update's partials + totals (disjoint regions)
    ALLOC(w.red, (size_t)residual_blocks(w.N) + 8 + 3 * (size_t)update_blocks(g.nx, g.ny) + 8);
    ALLOC(w.counters, 8);
    ALLOC(w.hist, (size_t)kHistSlots * kHistStride);
    if (!beta.empty()) {
        ALLOC(w.beta, N);
        CUDA_TRY(j, cudaMemcpyAsync(w.beta, beta.data(), N * sizeof(double), cudaMemcpyHostToDevice, j->stream));
    }
#undef ALLOC
    launch_mask_idx(w.node2x, (int)nxy, w.idx, j->stream);
    launch_mask_rows(w.node2x, g.nx, g.ny, w.rows, j->stream);
    launch_fill(w.c, (float)g.c0, nxy, j->stream);
    LAUNCHED(j, 3);
    CUDA_TRY(j, cudaMemsetAsync(w.counters, 0, 8 * sizeof(unsigned long long), j->stream));
    CUDA_TRY(j, cudaStreamSynchronize(j->stream));
    j->g = g;
    j->has_geom = true;
    return RBX_OK;
}

rbx_status rbx_mask(rbx_job *j, int *X_out, int *idx_dev)
{
    if (!j) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_mask before rbx_set_geometry");
    if (X_out) *X_out = j->w.X;
    if (idx_dev)
        CUDA_TRY(j, cudaMemcpyAsync(idx_dev, j->w.idx, sizeof(int) * j->w.X, cudaMemcpyDeviceToDevice, j->stream));
    return RBX_OK;
}

rbx_status rbx_set_model(rbx_job *j, const float *c_dev)
{
    if (!j || !c_dev) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_set_model before rbx_set_geometry");
    size_t nxy = (size_t)j->w.nx * j->w.ny;
    CUDA_TRY(j, cudaMemcpyAsync(j->w.c, c_dev, nxy * sizeof(float), cudaMemcpyDeviceToDevice, j->stream));
    CUDA_TRY(j, cudaMemsetAsync(j->w.counters + 5, 0, sizeof(unsigned long long), j->stream));
    launch_check_model(j->w.c, (int)nxy, j->w.counters + 5, j->stream);
    LAUNCHED(j, 1);
    unsigned long long bad = 0;
    CUDA_TRY(j, cudaMemcpyAsync(&bad, j->w.counters + 5, sizeof bad, cudaMemcpyDeviceToHost, j->stream));
    CUDA_TRY(j, cudaStreamSynchronize(j->stream));
    j->ns_valid = false;
    NEED(j, bad == 0, RBX_ENUMERIC, "sound speed must be finite and positive everywhere");
    return RBX_OK;
}

rbx_status rbx_set_absorption(rbx_job *j, const float *alpha0_dev, double y)
{
    if (!j) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_set_absorption before rbx_set_geometry");
    j->ns_valid = j->has_tables = false;
    if (!alpha0_dev) {
        j->lossy = false;
        return RBX_OK;
    }
    NEED(j, std::isfinite(y) && y > 0.0 && y < 2.0 && std::fabs(y - 1.0) > 1e-6, RBX_EINVAL,
         "power-law exponent y must lie in (0, 2) and differ from 1 (tan(pi y/2) is finite)");
    Workspace &w = j->w;
    const size_t nxy = (size_t)w.nx * w.ny;
    if (!w.alpha0) {
        if (dalloc(w.alpha0, nxy, j->stream) != cudaSuccess || dalloc(w.as64, nxy, j->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(j, RBX_ENOMEM, "device allocation of the absorption map failed");
        }
    }
    CUDA_TRY(j, cudaMemcpyAsync(w.alpha0, alpha0_dev, nxy * sizeof(float), cudaMemcpyDeviceToDevice, j->stream));
    CUDA_TRY(j, cudaMemsetAsync(w.counters + 5, 0, sizeof(unsigned long long), j->stream));
    launch_check_alpha(w.alpha0, (int)nxy, w.counters + 5, j->stream);
    LAUNCHED(j, 1);
    unsigned long long bad = 0;
    CUDA_TRY(j, cudaMemcpyAsync(&bad, w.counters + 5, sizeof bad, cudaMemcpyDeviceToHost, j->stream));
    CUDA_TRY(j, cudaStreamSynchronize(j->stream));
    NEED(j, bad == 0, RBX_EINVAL, "absorption coefficients must be finite and >= 0");
    j->lossy = true;
    j->abs_y = y;
    return RBX_OK;
}

rbx_status rbx_get_model(rbx_job *j, float *c_dev)
{
    if (!j || !c_dev) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_get_model before rbx_set_geometry");
    size_t nxy = (size_t)j->w.nx * j->w.ny;
    CUDA_TRY(j, cudaMemcpyAsync(c_dev, j->w.c, nxy * sizeof(float), cudaMemcpyDeviceToDevice, j->stream));
    return RBX_OK;
}

static Lossy lossy_of(const rbx_job *j)
{
    Lossy ab;
    if (j->lossy) {
        ab.alpha0 = j->w.alpha0;
        ab.as64 = j->w.as64;
        ab.y = j->abs_y;
    }
    return ab;
}

static rbx_status smooth(rbx_job *j, double f)
{
    int w = window_for(f, j->g.dx);
    if (j->ns_valid && j->ns_window == w && (!j->lossy || j->ns_freq == f)) return RBX_OK;
    launch_smooth_fields(j->g, j->w.c, w, j->w.tmp64, j->w.ns64, j->w.ns, j->w.fields, lossy_of(j), f, j->raw,
                         j->stream);
    LAUNCHED(j, j->lossy ? 5 : 3);
    j->ns_valid = true;
    j->ns_window = w;
    j->ns_freq = f;
    return RBX_OK;
}

static bool bad_freq(double f) { return !(std::isfinite(f) && f > 0); }

static RayParams ray_params(const rbx_job *j)
{
    const Workspace &w = j->w;
    RayParams p;
    p.N = w.N; p.X = w.X; p.nx = w.nx; p.ny = w.ny;
    p.dx = (float)j->g.dx; p.x0 = (float)j->g.x0; p.y0 = (float)j->g.y0;
    p.R = (float)j->g.ring_radius; p.ds = (float)j->g.ds; p.inv_dx = (float)(1.0 / j->g.dx);
    p.rmask = (float)j->g.mask_radius;
    p.maxs = max_steps(j->g);
    p.beta = w.beta;
    return p;
}

// Direct Green's function at the receivers: the fan's exit-angle interpolation, or secant
// linking of each pair on the current fields (rbx_set_linking), done once per trace and
// reused by every frequency.
static rbx_status direct_green(rbx_job *j, double f, float2 *out)
{
    Workspace &w = j->w;
    if (j->link_iters > 0) {
        if (!j->linked_valid) {
            launch_link_rays(w.fields, ray_params(j), w.exits, j->link_iters, w.linked, w.counters, j->lossy, j->raw,
                             j->stream);
            LAUNCHED(j, 1);
            j->linked_valid = true;
        }
        launch_green_linked(w.linked, w.N, f, j->g.c0, out, j->stream);
    } else {
        launch_direct_green(w.exits, w.N, w.beta, f, j->g.c0, out, w.counters, j->stream);
    }
    LAUNCHED(j, 1);
    return RBX_OK;
}

// The angular density array w.dg (step a4), formed when first needed after the tables changed:
// the FP32 back-projection and rbx_get_tables read it; the tensor-core operand synthesis forms
// the same values from the tables itself.
static rbx_status ensure_dgamma(rbx_job *j)
{
    if (j->dg_valid) return RBX_OK;
    launch_dgamma(j->w.tab, j->w.dg, j->w.N, j->w.X, j->stream);
    LAUNCHED(j, 1);
    j->dg_valid = true;
    return RBX_OK;
}

// The trace of step a2/a3 in three parts, so that the batched form can run the middle one
// for all its jobs as one grouped launch: the fields and the cleared tables, the ray trace
// with its rasteriser, and the tables' bookkeeping.
static rbx_status trace_begin(rbx_job *j, double f)
{
    Workspace &w = j->w;
    rbx_status st;
    if ((st = record(j, EV_START))) return st;
    j->ns_valid = false;   // recompute the fields for this model
    if ((st = smooth(j, f))) return st;
    if ((st = record(j, EV_FIELDS))) return st;
    CUDA_TRY(j, cudaMemsetAsync(w.tab, 0xff, sizeof(TabEntry) * (size_t)w.N * w.X, j->stream));
    CUDA_TRY(j, cudaMemsetAsync(w.counters, 0, 4 * sizeof(unsigned long long), j->stream));
    CUDA_TRY(j, cudaMemsetAsync(w.counters + 7, 0, sizeof(unsigned long long), j->stream));
    launch_uniform_radius(w.fields, ray_params(j), w.counters + 7, j->stream);
    LAUNCHED(j, 1);
    return RBX_OK;
}

static rbx_status trace_launch(rbx_job *j)
{
    Workspace &w = j->w;
    launch_trace_raster(w.fields, w.rows, w.tab, w.exits, ray_params(j), w.counters, j->lossy, j->raw, j->stream);
    LAUNCHED(j, 1);
    return RBX_OK;
}

static rbx_status trace_end(rbx_job *j)
{
    rbx_status st;
    j->linked_valid = j->dg_valid = false;
    if ((st = record(j, EV_TRACE))) return st;
    if (j->g.precision == RBX_FP32 && (st = ensure_dgamma(j))) return st;
    if ((st = record(j, EV_TABLES))) return st;
    j->has_tables = true;
    return RBX_OK;
}

rbx_status rbx_trace_rays(rbx_job *j, double f)
{
    if (!j) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_trace_rays before rbx_set_geometry");
    NEED(j, !bad_freq(f), RBX_EINVAL, "frequency must be finite and > 0");
    rbx_status st;
    if ((st = trace_begin(j, f))) return st;
    if ((st = trace_launch(j))) return st;
    return trace_end(j);
}

rbx_status rbx_set_tables(rbx_job *j, const float *T, const float *a, const float *gam, const uint8_t *K,
                          const float *exits)
{
    if (!j || !T || !a || !gam || !K || !exits) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_set_tables before rbx_set_geometry");
    Workspace &w = j->w;
    size_t n = (size_t)w.N * w.X;
    CUDA_TRY(j, cudaMemsetAsync(w.counters, 0, 4 * sizeof(unsigned long long), j->stream));
    launch_set_tables(T, a, gam, K, w.tab, n, w.counters, j->stream);
    j->linked_valid = j->dg_valid = false;
    CUDA_TRY(j, cudaMemcpyAsync(w.exits, exits, sizeof(float4) * (size_t)w.N * (w.N - 1), cudaMemcpyDeviceToDevice,
                                j->stream));
    LAUNCHED(j, 1);
    j->has_tables = true;
    return RBX_OK;
}

rbx_status rbx_get_tables(rbx_job *j, float *T, float *a, float *gam, uint8_t *K, float *dg, float *exits)
{
    if (!j) return RBX_EINVAL;
    NEED(j, j->has_tables, RBX_ESTATE, "rbx_get_tables before rbx_trace_rays or rbx_set_tables");
    Workspace &w = j->w;
    size_t n = (size_t)w.N * w.X;
    if (T || a || gam || K) {
        launch_get_tables(w.tab, T, a, gam, K, n, j->stream);
        LAUNCHED(j, 1);
    }
    if (dg) {
        rbx_status st = ensure_dgamma(j);
        if (st) return st;
        CUDA_TRY(j, cudaMemcpyAsync(dg, w.dg, sizeof(float) * n, cudaMemcpyDeviceToDevice, j->stream));
    }
    if (exits)
        CUDA_TRY(j, cudaMemcpyAsync(exits, w.exits, sizeof(float4) * (size_t)w.N * (w.N - 1), cudaMemcpyDeviceToDevice,
                                    j->stream));
    return RBX_OK;
}

rbx_status rbx_direct_green(rbx_job *j, double f, void *g_dev)
{
    if (!j || !g_dev) return RBX_EINVAL;
    NEED(j, j->has_tables, RBX_ESTATE, "rbx_direct_green before rbx_trace_rays or rbx_set_tables");
    NEED(j, !bad_freq(f), RBX_EINVAL, "frequency must be finite and > 0");
    if (j->link_iters > 0) {
        rbx_status st = smooth(j, f);   // the linked rays follow the smoothed map of f
        if (st) return st;
    }
    return direct_green(j, f, static_cast<float2 *>(g_dev));
}

// D = sum_x G_r G_e v on the current tables, into w.D (symmetric).
// The Born forward on the current tables with the weights in w.v. With both (tensor-core
// paths) the operand synthesis also writes the back-projection's planes for this frequency.
static rbx_status forward_core(rbx_job *j, double f, bool timed, bool both = false)
{
    Workspace &w = j->w;
    rbx_status st;
    if (j->g.precision != RBX_FP32 && w.tc.fwd_fused) {
        // the tuner's choice: the forward forms its operands from the tables; an update still
        // writes the back-projection's planes
        if (both) {
            launch_synth_bp_tc(w.tc, w.tab, f, j->g.c0, j->stream);
            LAUNCHED(j, 1);
        }
        if (timed && (st = record(j, EV_SYNTH_F))) return st;
        int splits = launch_forward_tc_fused(w.tc, w.tab, w.v, f, j->g.c0, w.part, j->stream);
        launch_forward_reduce(w.part, w.N, splits, w.D, j->stream);
        LAUNCHED(j, 2);
    } else if (j->g.precision != RBX_FP32) {
        if (both)
            launch_synth_both_tc(w.tc, w.tab, w.v, f, j->g.c0, j->stream);
        else
            launch_synth_fwd_tc(w.tc, w.tab, w.v, f, j->g.c0, j->stream);
        LAUNCHED(j, 1);
        if (timed && (st = record(j, EV_SYNTH_F))) return st;
        int splits = launch_forward_tc(w.tc, w.part, j->stream);
        launch_forward_reduce(w.part, w.N, splits, w.D, j->stream);
        LAUNCHED(j, 2);
    } else {
        launch_synth_fwd(w.tab, w.N, w.X, f, j->g.c0, w.G, j->stream);
        LAUNCHED(j, 1);
        if (timed && (st = record(j, EV_SYNTH_F))) return st;
        launch_forward_simt(w.G, w.v, w.N, w.X, w.fwd_splits, w.part, j->stream);
        launch_forward_reduce(w.part, w.N, w.fwd_splits, w.D, j->stream);
        LAUNCHED(j, 2);
    }
    if (timed && (st = record(j, EV_GEMM_F))) return st;
    return RBX_OK;
}

rbx_status rbx_forward(rbx_job *j, double f, const float *dm_dev, void *D_dev)
{
    if (!j || !dm_dev || !D_dev) return RBX_EINVAL;
    NEED(j, j->has_tables, RBX_ESTATE, "rbx_forward before rbx_trace_rays or rbx_set_tables");
    NEED(j, !bad_freq(f), RBX_EINVAL, "frequency must be finite and > 0");
    Workspace &w = j->w;
    launch_born_weights_dm(dm_dev, w.c, w.idx, w.X, f, j->g.dx * j->g.dx, lossy_of(j), w.v, j->stream);
    LAUNCHED(j, 1);
    rbx_status st = forward_core(j, f, false);
    if (st) return st;
    CUDA_TRY(j, cudaMemcpyAsync(D_dev, w.D, sizeof(float2) * (size_t)w.N * w.N, cudaMemcpyDeviceToDevice, j->stream));
    return RBX_OK;
}

rbx_status rbx_predict(rbx_job *j, double f, void *g_dev)
{
    if (!j || !g_dev) return RBX_EINVAL;
    NEED(j, j->has_tables, RBX_ESTATE, "rbx_predict before rbx_trace_rays or rbx_set_tables");
    NEED(j, !bad_freq(f), RBX_EINVAL, "frequency must be finite and > 0");
    Workspace &w = j->w;
    rbx_status st;
    if ((st = smooth(j, f))) return st;
    if ((st = direct_green(j, f, w.gdir))) return st;
    if (j->raw) {
        // integration on the non-smoothed map: the ray Green's function alone (Sec. 6.3.2)
        CUDA_TRY(j, cudaMemsetAsync(w.D, 0, sizeof(float2) * (size_t)w.N * w.N, j->stream));
    } else {
        launch_born_weights_rough(w.c, w.ns64, w.idx, w.X, f, j->g.dx * j->g.dx, lossy_of(j), w.v, j->stream);
        LAUNCHED(j, 1);
        if ((st = forward_core(j, f, false))) return st;
    }
    launch_add_offdiag(w.gdir, w.D, w.N, static_cast<float2 *>(g_dev), j->stream);
    LAUNCHED(j, 1);
    return RBX_OK;
}

rbx_status rbx_adjoint(rbx_job *j, double f, const void *R_dev, void *out_dev, int preconditioned)
{
    if (!j || !R_dev || !out_dev) return RBX_EINVAL;
    NEED(j, j->has_tables, RBX_ESTATE, "rbx_adjoint before rbx_trace_rays or rbx_set_tables");
    NEED(j, !bad_freq(f), RBX_EINVAL, "frequency must be finite and > 0");
    Workspace &w = j->w;
    launch_symmetrize(static_cast<const float2 *>(R_dev), w.N, w.Rs, j->stream);
    LAUNCHED(j, 1);
    if (preconditioned && j->g.precision != RBX_FP32) {
        launch_synth_bp_tc(w.tc, w.tab, f, j->g.c0, j->stream);
        launch_backproject_tc(w.tc, w.Rs, j->g.weight_mode, w.gpart, j->stream);
        launch_combine_adjoint(w.gpart, w.X, 0, j->g.weight_mode, 2.0, static_cast<float2 *>(out_dev), j->stream);
        LAUNCHED(j, 1);
    } else if (preconditioned) {
        rbx_status st = ensure_dgamma(j);
        if (st) return st;
        launch_synth_bp(w.tab, w.dg, w.N, w.X, f, j->g.c0, w.U, w.kap, j->stream);
        launch_backproject_simt(w.U, w.kap, w.Rs, w.N, w.X, 0, w.gpart, j->stream);
        launch_combine_adjoint(w.gpart, w.X, 0, j->g.weight_mode, 2.0, static_cast<float2 *>(out_dev), j->stream);
    } else {
        double om = 2 * 3.14159265358979323846 * f;
        launch_synth_fwd(w.tab, w.N, w.X, f, j->g.c0, w.G, j->stream);
        launch_backproject_simt(w.G, nullptr, w.Rs, w.N, w.X, 1, w.gpart, j->stream);
        if (j->lossy)
            launch_combine_adjoint_lossy(w.gpart, w.c, w.idx, w.X, f, j->g.dx * j->g.dx, lossy_of(j),
                                         static_cast<float2 *>(out_dev), j->stream);
        else
            launch_combine_adjoint(w.gpart, w.X, 1, j->g.weight_mode, om * om * j->g.dx * j->g.dx,
                                   static_cast<float2 *>(out_dev), j->stream);
    }
    LAUNCHED(j, 3);
    return RBX_OK;
}

// Steps a5-a9 queued on the job's stream with no host interaction (capturable into a CUDA
// graph); the update's scalar results are copied into device history slot `slot`.
// Steps a5-a8 of one frequency f on the current tables and the update kernel in `mode`
// (0: apply this frequency's step; 1/2/3: start / add to / finish a frequency set's sum).
static rbx_status enqueue_freq(rbx_job *j, double f, double df, const float2 *data, int mode)
{
    Workspace &w = j->w;
    rbx_status st;
    if ((st = direct_green(j, f, w.gdir))) return st;
    if ((st = record(j, EV_GDIR))) return st;
    if (j->raw) {
        // integration on the non-smoothed map: the residual is the ray Green's function alone
        CUDA_TRY(j, cudaMemsetAsync(w.D, 0, sizeof(float2) * (size_t)w.N * w.N, j->stream));
        if ((st = record(j, EV_SYNTH_F))) return st;
        if ((st = record(j, EV_GEMM_F))) return st;
    } else {
        launch_born_weights_rough(w.c, w.ns64, w.idx, w.X, f, j->g.dx * j->g.dx, lossy_of(j), w.v, j->stream);
        LAUNCHED(j, 1);
        if ((st = forward_core(j, f, true, true))) return st;
    }
    launch_residual(w.gdir, w.D, data, w.N, nullptr, w.Rs, w.red, j->stream);
    LAUNCHED(j, 2);
    if ((st = record(j, EV_RESID))) return st;
    if (j->g.precision != RBX_FP32) {
        if (j->raw) {   // otherwise the forward's synthesis wrote these planes
            launch_synth_bp_tc(w.tc, w.tab, f, j->g.c0, j->stream);
            LAUNCHED(j, 1);
        }
        if ((st = record(j, EV_SYNTH_B))) return st;
        launch_backproject_tc(w.tc, w.Rs, j->g.weight_mode, w.gpart, j->stream);
        LAUNCHED(j, 3);
    } else {
        if ((st = ensure_dgamma(j))) return st;
        launch_synth_bp(w.tab, w.dg, w.N, w.X, f, j->g.c0, w.U, w.kap, j->stream);
        LAUNCHED(j, 1);
        if ((st = record(j, EV_SYNTH_B))) return st;
        launch_backproject_simt(w.U, w.kap, w.Rs, w.N, w.X, 0, w.gpart, j->stream);
        LAUNCHED(j, 1);
    }
    if ((st = record(j, EV_GEMM_B))) return st;
    const int roff = residual_blocks(w.N) + 8;
    launch_update(w.gpart, w.node2x, w.nx, w.ny, w.X, j->g.weight_mode, f, df, j->g.tau, j->g.c0, w.c, w.red + roff,
                  w.counters, lossy_of(j), w.dmacc, mode, j->stream);
    LAUNCHED(j, 2);
    return RBX_OK;
}

static rbx_status enqueue_update(rbx_job *j, double f, double df, const float2 *data, bool traced, int slot)
{
    Workspace &w = j->w;
    rbx_status st;
    if (!traced && (st = record(j, EV_TABLES))) return st;
    if ((st = smooth(j, f))) return st;
    CUDA_TRY(j, cudaMemsetAsync(w.counters + 1, 0, sizeof(unsigned long long), j->stream));
    CUDA_TRY(j, cudaMemsetAsync(w.counters + 4, 0, sizeof(unsigned long long), j->stream));
    if ((st = enqueue_freq(j, f, df, data, 0))) return st;
    const int roff = residual_blocks(w.N) + 8;
    launch_snapshot(w.red + residual_blocks(w.N), w.red + roff + 3 * update_blocks(w.nx, w.ny), w.counters,
                    w.tc.err, (unsigned long long)w.N * w.X, w.hist + (size_t)slot * kHistStride, j->stream);
    LAUNCHED(j, 1);
    if ((st = record(j, EV_UPDATE))) return st;
    j->ns_valid = false;   // the model changed
    return RBX_OK;
}

// Scalar results of history slot `slot` as an rbx_stats (synchronises); returns the
// status the update ended with.
static rbx_status read_stats(rbx_job *j, int slot, rbx_stats *out, bool traced, bool timing)
{
    Workspace &w = j->w;
    double h[kHistStride];
    CUDA_TRY(j, cudaMemcpyAsync(h, w.hist + (size_t)slot * kHistStride, sizeof h, cudaMemcpyDeviceToHost, j->stream));
    CUDA_TRY(j, cudaStreamSynchronize(j->stream));
    if (out) {
        std::memset(out, 0, sizeof *out);
        out->resid_norm2 = h[0];
        out->rms_dc = std::sqrt(h[1] / w.X);
        out->max_abs_dc = h[2];
        out->dm_norm = std::sqrt(h[3]);
        out->n_uncovered = (long long)h[4];
        out->n_clamped = (long long)h[5];
        if (timing) {
            int t0 = traced ? EV_START : EV_TABLES;
            out->ms_trace = traced ? elapsed(j, EV_START, EV_TABLES) : 0.f;
            out->ms_forward = elapsed(j, EV_TABLES, EV_RESID);
            out->ms_backproj = elapsed(j, EV_RESID, EV_UPDATE);
            out->ms_total = elapsed(j, t0, EV_UPDATE);
            if (traced) {
                out->ms_kernel[RBX_K_FIELDS] = elapsed(j, EV_START, EV_FIELDS);
                out->ms_kernel[RBX_K_TRACE] = elapsed(j, EV_FIELDS, EV_TRACE);
            }
            out->ms_kernel[RBX_K_TABLES] =
                (traced ? elapsed(j, EV_TRACE, EV_TABLES) : 0.f) + elapsed(j, EV_TABLES, EV_GDIR);
            out->ms_kernel[RBX_K_SYNTH_FWD] = elapsed(j, EV_GDIR, EV_SYNTH_F);
            out->ms_kernel[RBX_K_GEMM_FWD] = elapsed(j, EV_SYNTH_F, EV_GEMM_F);
            out->ms_kernel[RBX_K_SYNTH_BP] = elapsed(j, EV_RESID, EV_SYNTH_B);
            out->ms_kernel[RBX_K_GEMM_BP] = elapsed(j, EV_SYNTH_B, EV_GEMM_B);
            out->ms_kernel[RBX_K_UPDATE] = elapsed(j, EV_GEMM_F, EV_RESID) + elapsed(j, EV_GEMM_B, EV_UPDATE);
        }
    }
    NEED(j, h[10] == 0, RBX_ETIMEOUT, "a tensor-core kernel's bounded wait gave up");
    NEED(j, h[8] == 0, RBX_ENUMERIC, "non-finite or non-positive updated squared slowness");
    NEED(j, h[6] == 0, RBX_ENUMERIC, "a ray did not reach the ring within the step limit");
    NEED(j, h[7] == 0, RBX_ECUDA, "table compare-and-swap exceeded its iteration bound");
    return RBX_OK;
}

// Status of a whole sweep: the first failing update among slots 0..nf-1 decides it (a later
// update starts from the kept model and may itself succeed); `out` gets the last slot.
static rbx_status read_sweep(rbx_job *j, int nf, rbx_stats *out)
{
    Workspace &w = j->w;
    std::vector<double> h((size_t)nf * kHistStride);
    CUDA_TRY(j, cudaMemcpyAsync(h.data(), w.hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost, j->stream));
    CUDA_TRY(j, cudaStreamSynchronize(j->stream));
    for (int s = 0; s < nf - 1; s++) {
        const double *hs = h.data() + (size_t)s * kHistStride;
        if (hs[10] != 0 || hs[8] != 0 || hs[6] != 0 || hs[7] != 0) {
            rbx_status st = read_stats(j, s, nullptr, true, false);
            if (st != RBX_OK) {
                char msg[64];
                std::snprintf(msg, sizeof msg, " (update %d of %d)", s + 1, nf);
                std::string keep = j->err + msg;
                if (out) read_stats(j, nf - 1, out, true, false);
                j->err = keep;
                return st;
            }
        }
    }
    return read_stats(j, nf - 1, out, true, false);
}

static rbx_status update_core(rbx_job *j, double f, double df, const float2 *data, rbx_stats *out, bool traced)
{
    rbx_status st = enqueue_update(j, f, df, data, traced, 0);
    if (st) return st;
    return read_stats(j, 0, out, traced, true);
}

rbx_status rbx_update_from_tables(rbx_job *j, double f, double df, const void *data_dev, rbx_stats *out)
{
    if (!j || !data_dev) return RBX_EINVAL;
    NEED(j, j->has_tables, RBX_ESTATE, "rbx_update_from_tables before rbx_trace_rays or rbx_set_tables");
    NEED(j, !bad_freq(f) && std::isfinite(df) && df > 0, RBX_EINVAL, "frequency and spacing must be finite and > 0");
    long long l0 = j->launches;
    rbx_status st = update_core(j, f, df, static_cast<const float2 *>(data_dev), out, false);
    if (out) out->n_launches = j->launches - l0;
    return st;
}

rbx_status rbx_update_frequency(rbx_job *j, double f, double df, const void *data_dev, rbx_stats *out)
{
    if (!j || !data_dev) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_update_frequency before rbx_set_geometry");
    NEED(j, !bad_freq(f) && std::isfinite(df) && df > 0, RBX_EINVAL, "frequency and spacing must be finite and > 0");
    long long l0 = j->launches;
    rbx_status st = rbx_trace_rays(j, f);
    if (st) return st;
    st = update_core(j, f, df, static_cast<const float2 *>(data_dev), out, true);
    if (out) out->n_launches = j->launches - l0;
    return st;
}

rbx_status rbx_set_linking(rbx_job *j, int max_rays)
{
    if (!j) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_set_linking before rbx_set_geometry");
    NEED(j, max_rays >= 0 && max_rays <= 32, RBX_EINVAL, "linking takes 0 (off) to 32 new rays per pair");
    if (max_rays > 0 && !j->w.linked) {
        if (dalloc(j->w.linked, (size_t)j->w.N * j->w.N, j->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(j, RBX_ENOMEM, "device allocation of the linked rays failed");
        }
    }
    j->link_iters = max_rays;
    j->linked_valid = false;
    return RBX_OK;
}

rbx_status rbx_set_integration(rbx_job *j, int mode)
{
    if (!j) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_set_integration before rbx_set_geometry");
    NEED(j, mode == 0 || mode == 1, RBX_EINVAL, "integration mode must be 0 (smoothed) or 1 (non-smoothed)");
    j->raw = mode == 1;
    j->ns_valid = j->has_tables = false;
    return RBX_OK;
}

rbx_status rbx_update_set(rbx_job *j, const double *freqs, int nf, double df, const void *data_dev, rbx_stats *out)
{
    if (!j || !freqs || !data_dev || nf < 1) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_update_set before rbx_set_geometry");
    NEED(j, nf <= 16, RBX_EINVAL, "at most 16 frequencies per set");
    NEED(j, std::isfinite(df) && df > 0, RBX_EINVAL, "frequency spacing must be finite and > 0");
    for (int k = 0; k < nf; k++) NEED(j, !bad_freq(freqs[k]), RBX_EINVAL, "frequencies must be finite and > 0");
    if (nf == 1) return rbx_update_frequency(j, freqs[0], df, data_dev, out);
    Workspace &w = j->w;
    long long l0 = j->launches;
    if (!w.dmacc && dalloc(w.dmacc, (size_t)w.X, j->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(j, RBX_ENOMEM, "device allocation of the set accumulator failed");
    }
    // one trace for the set, on the map smoothed (and dispersed) for its first frequency
    rbx_status st = rbx_trace_rays(j, freqs[0]);
    if (st) return st;
    CUDA_TRY(j, cudaMemsetAsync(w.counters + 1, 0, sizeof(unsigned long long), j->stream));
    CUDA_TRY(j, cudaMemsetAsync(w.counters + 4, 0, sizeof(unsigned long long), j->stream));
    const size_t nn = (size_t)w.N * w.N;
    const int nb = residual_blocks(w.N), roff = nb + 8;
    for (int k = 0; k < nf; k++) {
        const float2 *d = static_cast<const float2 *>(data_dev) + (size_t)k * nn;
        if ((st = enqueue_freq(j, freqs[k], df, d, k == 0 ? 1 : (k < nf - 1 ? 2 : 3)))) return st;
        launch_acc_scalar(w.red + nb, w.red + nb + 4, k == 0, j->stream);
        LAUNCHED(j, 1);
    }
    launch_snapshot(w.red + nb + 4, w.red + roff + 3 * update_blocks(w.nx, w.ny), w.counters, w.tc.err,
                    (unsigned long long)w.N * w.X, w.hist, j->stream);
    LAUNCHED(j, 1);
    if ((st = record(j, EV_UPDATE))) return st;
    j->ns_valid = false;
    st = read_stats(j, 0, out, true, false);
    if (out) out->n_launches = j->launches - l0;
    return st;
}

rbx_status rbx_update_frequency_host(rbx_job *j, double f, double df, const void *data_host, float *c_out_host,
                                     rbx_stats *out)
{
    if (!j || !data_host) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_update_frequency_host before rbx_set_geometry");
    NEED(j, !bad_freq(f) && std::isfinite(df) && df > 0, RBX_EINVAL, "frequency and spacing must be finite and > 0");
    if (!j->copy_stream) {
        CUDA_TRY(j, cudaStreamCreateWithFlags(&j->copy_stream, cudaStreamNonBlocking));
        CUDA_TRY(j, cudaEventCreateWithFlags(&j->ev_in_free, cudaEventDisableTiming));
        CUDA_TRY(j, cudaEventCreateWithFlags(&j->ev_in_ready, cudaEventDisableTiming));
    }
    // The data's copy runs on the copy stream beside the trace (which does not read it), after
    // the work already queued on the job's stream, which may still read the previous data.
    size_t nn = (size_t)j->w.N * j->w.N;
    CUDA_TRY(j, cudaEventRecord(j->ev_in_free, j->stream));
    CUDA_TRY(j, cudaStreamWaitEvent(j->copy_stream, j->ev_in_free, 0));
    CUDA_TRY(j, cudaMemcpyAsync(j->w.data, data_host, sizeof(float2) * nn, cudaMemcpyHostToDevice, j->copy_stream));
    CUDA_TRY(j, cudaEventRecord(j->ev_in_ready, j->copy_stream));
    const long long l0 = j->launches;
    rbx_status st = rbx_trace_rays(j, f);
    if (st) {
        cudaStreamSynchronize(j->copy_stream);   // the copy still reads data_host
        return st;
    }
    CUDA_TRY(j, cudaStreamWaitEvent(j->stream, j->ev_in_ready, 0));
    st = enqueue_update(j, f, df, j->w.data, true, 0);
    if (st) {
        cudaStreamSynchronize(j->stream);
        return st;
    }
    if (c_out_host) {   // queued before the statistics' read, so that one wait covers both
        size_t nxy = (size_t)j->w.nx * j->w.ny;
        CUDA_TRY(j, cudaMemcpyAsync(c_out_host, j->w.c, sizeof(float) * nxy, cudaMemcpyDeviceToHost, j->stream));
    }
    st = read_stats(j, 0, out, true, true);
    if (out) out->n_launches = j->launches - l0;
    return st;
}

// rbx_update_frequency_async in two halves around the ray trace's launch (the batched form's
// grouped trace goes between them).
static rbx_status update_async_begin(rbx_job *j, double f, double df, const void *data_dev, int slot)
{
    if (!j || !data_dev) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_update_frequency_async before rbx_set_geometry");
    NEED(j, !bad_freq(f) && std::isfinite(df) && df > 0, RBX_EINVAL, "frequency and spacing must be finite and > 0");
    NEED(j, slot >= 0 && slot < kHistSlots, RBX_EINVAL, "stats slot must be in [0, 64)");
    j->slot_l0 = j->launches;
    if (j->slot_ev) j->evp = j->slot_ev + (size_t)slot * EV_COUNT;   // this update's own events
    rbx_status st = trace_begin(j, f);
    if (st) j->evp = j->ev;
    return st;
}

static rbx_status update_async_end(rbx_job *j, double f, double df, const void *data_dev, int slot)
{
    rbx_status st = trace_end(j);
    if (!st) st = enqueue_update(j, f, df, static_cast<const float2 *>(data_dev), true, slot);
    j->evp = j->ev;
    j->slot_launches[slot] = j->launches - j->slot_l0;
    return st;
}

rbx_status rbx_update_frequency_async(rbx_job *j, double f, double df, const void *data_dev, int slot)
{
    rbx_status st = update_async_begin(j, f, df, data_dev, slot);
    if (st) return st;
    if ((st = trace_launch(j))) {
        j->evp = j->ev;
        return st;
    }
    return update_async_end(j, f, df, data_dev, slot);
}

rbx_status rbx_set_slot_timing(rbx_job *j, int on)
{
    if (!j) return RBX_EINVAL;
    if (!on) {
        if (j->slot_ev) {
            CUDA_TRY(j, cudaStreamSynchronize(j->stream));
            for (int k = 0; k < kHistSlots * EV_COUNT; k++)
                if (j->slot_ev[k]) cudaEventDestroy(j->slot_ev[k]);
            delete[] j->slot_ev;
            j->slot_ev = nullptr;
        }
        return RBX_OK;
    }
    if (j->slot_ev) return RBX_OK;
    j->slot_ev = new (std::nothrow) cudaEvent_t[(size_t)kHistSlots * EV_COUNT]();
    if (!j->slot_ev) return fail(j, RBX_ENOMEM, "host allocation of the slot events failed");
    for (int k = 0; k < kHistSlots * EV_COUNT; k++) {
        if (cudaEventCreate(&j->slot_ev[k]) != cudaSuccess) {
            cudaGetLastError();
            for (int q = 0; q < k; q++) cudaEventDestroy(j->slot_ev[q]);
            delete[] j->slot_ev;
            j->slot_ev = nullptr;
            return fail(j, RBX_ECUDA, "creation of the slot events failed");
        }
    }
    return RBX_OK;
}

rbx_status rbx_get_stats(rbx_job *j, int slot, rbx_stats *out)
{
    if (!j) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_get_stats before rbx_set_geometry");
    NEED(j, slot >= 0 && slot < kHistSlots, RBX_EINVAL, "stats slot must be in [0, 64)");
    if (!j->slot_ev) return read_stats(j, slot, out, true, false);
    j->evp = j->slot_ev + (size_t)slot * EV_COUNT;
    rbx_status st = read_stats(j, slot, out, true, true);
    j->evp = j->ev;
    if (out) out->n_launches = j->slot_launches[slot];
    return st;
}

static double sweep_df(const double *freqs, int nf, int n)
{
    if (nf == 1) return 1e5;
    if (n == 0) return freqs[1] - freqs[0];
    if (n == nf - 1) return freqs[nf - 1] - freqs[nf - 2];
    return 0.5 * (freqs[n + 1] - freqs[n - 1]);
}

// The whole sweep of one job on its stream, update n writing stats slot n.
static rbx_status enqueue_sweep(rbx_job *j, const double *freqs, int nf, const void *data_dev)
{
    size_t nn = (size_t)j->w.N * j->w.N;
    for (int n = 0; n < nf; n++) {
        double df = sweep_df(freqs, nf, n);
        NEED(j, std::isfinite(df) && df > 0, RBX_EINVAL, "frequencies must increase");
        const float2 *d = static_cast<const float2 *>(data_dev) + (size_t)n * nn;
        rbx_status st = rbx_update_frequency_async(j, freqs[n], df, d, n);
        if (st) return st;
    }
    return RBX_OK;
}

rbx_status rbx_batch_run(rbx_job *const *jobs, int n, const double *const *freqs, const int *nf,
                         const void *const *data_dev, int use_graph, rbx_stats *last, float *ms_total)
{
    if (!jobs || n < 1 || !freqs || !nf || !data_dev) return RBX_EINVAL;
    for (int i = 0; i < n; i++) {
        if (!jobs[i] || !freqs[i] || !data_dev[i] || nf[i] < 1) return RBX_EINVAL;
        NEED(jobs[i], jobs[i]->has_geom, RBX_ESTATE, "rbx_batch_run on a job without geometry");
        NEED(jobs[i], nf[i] <= kHistSlots, RBX_EINVAL, "at most 64 frequencies per job in a batch");
        for (int k = 0; k < i; k++)
            NEED(jobs[i], jobs[k] != jobs[i], RBX_EINVAL, "a job appears twice in the batch");
    }
    rbx_job *j0 = jobs[0];
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t *streams = new (std::nothrow) cudaStream_t[n]();
    cudaEvent_t *joins = new (std::nothrow) cudaEvent_t[n]();
    cudaStream_t *saved = new (std::nothrow) cudaStream_t[n]();
    rbx_status st = RBX_OK;
    bool capturing = false;
    if (!streams || !joins || !saved) st = RBX_ENOMEM;
    // the grouped trace needs one instantiation of the trace for all jobs
    bool grouped = (use_graph & RBX_BATCH_GROUPED) != 0;
    for (int i = 1; i < n; i++)
        if (jobs[i]->lossy != j0->lossy || jobs[i]->raw != j0->raw) grouped = false;
    int maxnf = 0, max_ny = 0, gblocks = 0;
    std::vector<TraceGroup> groups;   // launches of step q: groups[gfirst[q] .. gfirst[q + 1])
    std::vector<int> gfirst;
    int *next_dev = nullptr;          // one work counter per launch
    cudaEvent_t trev = nullptr;
#define BTRY(call)                                                                                       \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess && st == RBX_OK) st = fail(j0, RBX_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
    if (st == RBX_OK) {
        BTRY(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
        BTRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        BTRY(cudaEventCreate(&t0));
        BTRY(cudaEventCreate(&t1));
        for (int i = 0; i < n && st == RBX_OK; i++) {
            BTRY(cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking));
            BTRY(cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming));
            // wait for work already queued on the job's own stream, then run on the batch stream
            BTRY(cudaStreamSynchronize(jobs[i]->stream));
            saved[i] = jobs[i]->stream;
            jobs[i]->stream = streams[i];
        }
    }
    if (st == RBX_OK && grouped) {
        // work lists of the grouped traces, one per sweep step q: the jobs still sweeping,
        // longest in-mask ray paths (mask radius over step length) first, so that the list
        // ends with the cheapest items; kMaxGroup jobs per launch
        std::vector<int> order(n);
        for (int i = 0; i < n; i++) {
            order[i] = i;
            maxnf = std::max(maxnf, nf[i]);
            max_ny = std::max(max_ny, jobs[i]->w.ny);
        }
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return jobs[a]->g.mask_radius / jobs[a]->g.ds > jobs[b]->g.mask_radius / jobs[b]->g.ds;
        });
        for (int q = 0; q < maxnf; q++) {
            gfirst.push_back((int)groups.size());
            for (int i : order) {
                if (q >= nf[i]) continue;
                if (groups.size() == (size_t)gfirst.back() || groups.back().njobs == kMaxGroup) {
                    groups.emplace_back();
                    std::memset(&groups.back(), 0, sizeof(TraceGroup));
                }
                TraceGroup &gr = groups.back();
                const Workspace &w = jobs[i]->w;
                TraceJob &t = gr.j[gr.njobs++];
                t.F = w.fields; t.rows = w.rows; t.tab = w.tab; t.exits = w.exits; t.counters = w.counters;
                t.p = ray_params(jobs[i]);
                t.item0 = gr.total;
                gr.total += trace_items(w.N, &t.nwarps);
            }
        }
        gfirst.push_back((int)groups.size());
        gblocks = trace_grouped_blocks(j0->lossy, j0->raw, max_ny);
        if (gblocks < 1) st = fail(j0, RBX_ECUDA, "no resident block for the grouped trace");
        BTRY(cudaMalloc(&next_dev, sizeof(int) * groups.size()));
        BTRY(cudaEventCreateWithFlags(&trev, cudaEventDisableTiming));
    }
    if (st == RBX_OK) {
        if (use_graph & RBX_BATCH_GRAPH) {
            BTRY(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
            capturing = st == RBX_OK;
        } else {
            BTRY(cudaEventRecord(t0, origin));
        }
        BTRY(cudaEventRecord(fork, origin));
        if (!grouped) {
            for (int i = 0; i < n && st == RBX_OK; i++) {
                BTRY(cudaStreamWaitEvent(streams[i], fork, 0));
                if (st == RBX_OK) {
                    rbx_status s2 = enqueue_sweep(jobs[i], freqs[i], nf[i], data_dev[i]);
                    if (s2 != RBX_OK) {
                        st = s2;
                        if (jobs[i] != j0) j0->err = jobs[i]->err;
                    }
                }
                BTRY(cudaEventRecord(joins[i], streams[i]));
                BTRY(cudaStreamWaitEvent(origin, joins[i], 0));
            }
        } else {
            // Lock-step by sweep step: each job queues its fields and cleared tables on its own
            // stream, one persistent launch on the origin stream traces all of them, and each
            // job queues the rest of its update after it. Only the trace is shared: a job's
            // contractions and update overlap the other jobs' and its next step's fields.
            for (int i = 0; i < n; i++) BTRY(cudaStreamWaitEvent(streams[i], fork, 0));
            auto job_fail = [&](int i, rbx_status s2) {
                if (st == RBX_OK) {
                    st = s2;
                    if (jobs[i] != j0) j0->err = jobs[i]->err;
                }
            };
            for (int q = 0; q < maxnf && st == RBX_OK; q++) {
                int first = -1;
                for (int i = 0; i < n && st == RBX_OK; i++) {
                    if (q >= nf[i]) continue;
                    if (first < 0) first = i;
                    const double df = sweep_df(freqs[i], nf[i], q);
                    if (!(std::isfinite(df) && df > 0)) {
                        job_fail(i, fail(jobs[i], RBX_EINVAL, "frequencies must increase"));
                        break;
                    }
                    const float2 *d = static_cast<const float2 *>(data_dev[i]) + (size_t)q * jobs[i]->w.N * jobs[i]->w.N;
                    rbx_status s2 = update_async_begin(jobs[i], freqs[i][q], df, d, q);
                    if (s2 != RBX_OK) job_fail(i, s2);
                    BTRY(cudaEventRecord(joins[i], streams[i]));
                    BTRY(cudaStreamWaitEvent(origin, joins[i], 0));
                }
                if (st != RBX_OK) break;
                for (int k = gfirst[q]; k < gfirst[q + 1] && st == RBX_OK; k++) {
                    BTRY(cudaMemsetAsync(next_dev + k, 0, sizeof(int), origin));
                    launch_trace_grouped(groups[k], max_ny, gblocks, next_dev + k, j0->lossy, j0->raw, origin);
                    BTRY(cudaGetLastError());
                    jobs[first]->launches += 1;   // one launch for up to kMaxGroup jobs' traces
                }
                BTRY(cudaEventRecord(trev, origin));
                for (int i = 0; i < n && st == RBX_OK; i++) {
                    if (q >= nf[i]) continue;
                    BTRY(cudaStreamWaitEvent(streams[i], trev, 0));
                    const double df = sweep_df(freqs[i], nf[i], q);
                    const float2 *d = static_cast<const float2 *>(data_dev[i]) + (size_t)q * jobs[i]->w.N * jobs[i]->w.N;
                    rbx_status s2 = update_async_end(jobs[i], freqs[i][q], df, d, q);
                    if (s2 != RBX_OK) job_fail(i, s2);
                }
            }
            for (int i = 0; i < n; i++) {
                jobs[i]->evp = jobs[i]->ev;
                BTRY(cudaEventRecord(joins[i], streams[i]));
                BTRY(cudaStreamWaitEvent(origin, joins[i], 0));
            }
        }
        if (capturing) {
            cudaError_t e = cudaStreamEndCapture(origin, &graph);
            if (e != cudaSuccess && st == RBX_OK) st = fail(j0, RBX_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
            if (st == RBX_OK) BTRY(cudaGraphInstantiate(&exec, graph, 0));
            if (st == RBX_OK) {
                BTRY(cudaEventRecord(t0, origin));
                BTRY(cudaGraphLaunch(exec, origin));
            }
        }
        BTRY(cudaEventRecord(t1, origin));
        BTRY(cudaStreamSynchronize(origin));
    }
    if (st == RBX_OK && ms_total) BTRY(cudaEventElapsedTime(ms_total, t0, t1));
    for (int i = 0; i < n; i++) {
        if (streams && saved && streams[i] && jobs[i]->stream == streams[i]) jobs[i]->stream = saved[i];
        jobs[i]->ns_valid = false;
    }
    if (st == RBX_OK) {
        for (int i = 0; i < n && st == RBX_OK; i++) {
            rbx_job *j = jobs[i];
            rbx_stats tmp;
            rbx_status s2 = read_sweep(j, nf[i], last ? &last[i] : &tmp);
            if (s2 != RBX_OK) {
                st = s2;
                if (j != j0) j0->err = j->err;
            }
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (int i = 0; i < n; i++) {
        if (streams && streams[i]) cudaStreamDestroy(streams[i]);
        if (joins && joins[i]) cudaEventDestroy(joins[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (trev) cudaEventDestroy(trev);
    if (next_dev) cudaFree(next_dev);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (origin) cudaStreamDestroy(origin);
    delete[] streams;
    delete[] joins;
    delete[] saved;
#undef BTRY
    return st;
}

}  // extern "C"

// ---------------------------------------------------------------- hooks for the server (C++)
namespace rbx {
rbx_status job_enqueue_sweep(rbx_job *j, const double *freqs, int nf, const void *data_dev)
{
    for (int n = 0; n < nf; n++)
        if (!(std::isfinite(freqs[n]) && freqs[n] > 0)) return fail(j, RBX_EINVAL, "frequencies must be finite and > 0");
    NEED(j, nf <= kHistSlots, RBX_EINVAL, "at most 64 frequencies per request");
    return enqueue_sweep(j, freqs, nf, data_dev);
}
rbx_status job_read_sweep(rbx_job *j, int nf, rbx_stats *last) { return read_sweep(j, nf, last); }
cudaStream_t job_stream(const rbx_job *j) { return j->stream; }
float *job_model(rbx_job *j) { return j->w.c; }

// Upper estimate of the device bytes one job needs (admission control).
size_t job_bytes_estimate(const rbx_geometry &g, int nf)
{
    const double r = g.mask_radius / g.dx;
    const size_t X = (size_t)(3.14159265358979 * r * r + 6.3 * r + 16);
    const size_t N = (size_t)g.n_xducers, NX = N * X, nxy = (size_t)g.nx * g.ny, NN = N * N;
    size_t b = NX * (16 + 4 + 8);                                 // tables, angular density, G
    if (g.precision == RBX_FP32) b += NX * 16;                    // U, kappa
    else {
        const size_t Np = (N + 127) / 128 * 128, Xk = (X + 63) / 64 * 64, Xm = (X + 127) / 128 * 128;
        const size_t m = g.precision == RBX_BF16X3 ? 2 : 1;
        b += m * (4 * Np * Xk + 6 * Xm * Np + 2 * Np * Np) * 2 + (Np / 128) * Xm * 8;
    }
    b += nxy * (4 + 4 + 8 + 8 + 32 + 4 + 4) + N * (N - 1) * 16 + NN * 8 * 5 + 64 * NN * 8 + X * 24;
    b += (size_t)nf * NN * 8 + nxy * 4 + (1u << 20);              // data, initial model, slack
    return b;
}
}  // namespace rbx

extern "C" {

int rbx_autotune(int mode) { return set_autotune(mode); }

rbx_status rbx_get_tuning(const rbx_job *j, int *fwd_splits, int *candidates_timed)
{
    if (!j) return RBX_EINVAL;
    if (fwd_splits) *fwd_splits = j->g.precision == RBX_FP32 ? j->w.fwd_splits : j->w.tc.fwd_splits;
    if (candidates_timed) *candidates_timed = j->w.tc.tuned;
    return RBX_OK;
}

rbx_status rbx_get_tuning_times(const rbx_job *j, float *ms, int *fused)
{
    if (!j) return RBX_EINVAL;
    if (ms)
        for (int k = 0; k < 4; k++) ms[k] = j->w.tc.tune_ms[k];
    if (fused) *fused = j->w.tc.fwd_fused ? 1 : 0;
    return RBX_OK;
}

rbx_status rbx_selftest_bounded_wait(int *timed_out)
{
    if (!timed_out) return RBX_EINVAL;
    *timed_out = 0;
    unsigned *flag = nullptr, h = 0;
    if (cudaMalloc(&flag, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return RBX_ENOMEM;
    }
    rbx_status st = RBX_OK;
    if (cudaMemset(flag, 0, sizeof(unsigned)) != cudaSuccess) st = RBX_ECUDA;
    if (st == RBX_OK) {
        launch_wait_selftest(flag, 0);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(&h, flag, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = RBX_ECUDA;
    }
    cudaFree(flag);
    if (st == RBX_OK) *timed_out = h == 1u ? 1 : 0;
    return st;
}

rbx_status rbx_pool_usage(size_t *used, size_t *reserved, int trim)
{
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return RBX_ECUDA;
    if (trim) {
        if (cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(pool, 0) != cudaSuccess) return RBX_ECUDA;
    }
    uint64_t u = 0, r = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r) != cudaSuccess)
        return RBX_ECUDA;
    if (used) *used = (size_t)u;
    if (reserved) *reserved = (size_t)r;
    return RBX_OK;
}

rbx_status rbx_reconstruct(rbx_job *j, const double *freqs, int nf, const void *data_dev, rbx_stats *per_freq)
{
    if (!j || !freqs || nf < 1 || !data_dev) return RBX_EINVAL;
    NEED(j, j->has_geom, RBX_ESTATE, "rbx_reconstruct before rbx_set_geometry");
    size_t nn = (size_t)j->w.N * j->w.N;
    for (int n = 0; n < nf; n++) {
        double df;
        if (nf == 1) df = 1e5;
        else if (n == 0) df = freqs[1] - freqs[0];
        else if (n == nf - 1) df = freqs[nf - 1] - freqs[nf - 2];
        else df = 0.5 * (freqs[n + 1] - freqs[n - 1]);
        NEED(j, std::isfinite(df) && df > 0, RBX_EINVAL, "frequencies must increase");
        const float2 *d = static_cast<const float2 *>(data_dev) + (size_t)n * nn;
        rbx_status st = rbx_update_frequency(j, freqs[n], df, d, per_freq ? &per_freq[n] : nullptr);
        if (st) return st;
    }
    return RBX_OK;
}

}  // extern "C"
