/*
 * rbx.h -- C ABI of the GB300 ray-Born library: one preconditioned, Hessian-free
 * sound-speed update per frequency (Javaherian, arXiv 2211.00316).
 *
 * Geometry (Sec. 2.1): a 2-D square grid of nx x ny nodes, node (ix, iy) at
 * (x0 + ix dx, y0 + iy dx), arrays row-major [iy][ix]; N point transducers on a ring of
 * radius R centred at the origin, by default transducer e at R (cos 2 pi e/N, sin 2 pi e/N)
 * (rbx_set_geometry also takes other positions on the ring), each both emitter and receiver.
 * The reconstruction mask is |x| <= mask_radius (Sec. 6.3).
 *
 * Conventions shared by every call:
 *  - Pointers named *_dev are CUDA device pointers, *_host are host pointers. The caller
 *    owns every pointer it passes; the job owns only its internal workspaces.
 *  - Complex arrays are interleaved (re, im) float32. Data, residual and forward outputs
 *    are emitter-major N x N: element [e*N + r] holds g(omega, r, e) (receiver r, emitter e).
 *  - Frequencies are in Hz; omega = 2 pi f. The time-harmonic convention is that of
 *    Sec. 2.1 (p(omega) = int p(t) e^{+i omega t} dt): a delay T is the phase e^{+i omega T}.
 *  - Every call is asynchronous on the job's stream except those that fill an rbx_stats
 *    (they synchronise the stream before returning). A job is used by one host thread at a
 *    time. No call throws; each returns an rbx_status and rbx_last_error() describes the
 *    last failure of that job.
 *  - There is no CPU fallback: a call that cannot run its CUDA kernels fails with
 *    RBX_ECUDA.
 */
#ifndef RBX_H
#define RBX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbx_job rbx_job;

typedef enum {
    RBX_OK = 0,
    RBX_EINVAL = 1,    /* bad argument or geometry */
    RBX_ENOMEM = 2,    /* device allocation failed */
    RBX_ECUDA = 3,     /* a CUDA call or kernel failed (message in rbx_last_error) */
    RBX_ESTATE = 4,    /* call out of order, e.g. forward before trace_rays */
    RBX_ENUMERIC = 5,  /* non-finite input or a non-positive updated squared slowness */
    RBX_ETIMEOUT = 6   /* a bounded device-side wait gave up */
} rbx_status;

typedef enum {
    RBX_FP32 = 0,      /* FP32 SIMT contractions */
    RBX_BF16 = 1,      /* BF16 tensor-core contractions, FP32 accumulation */
    RBX_BF16X3 = 2     /* split BF16 (hi + lo, three products), FP32 accumulation */
} rbx_precision;

typedef struct {
    int nx, ny;             /* grid nodes */
    double dx;              /* grid spacing [m] */
    double x0, y0;          /* position of node (0,0) [m] */
    int n_xducers;          /* N >= 3 */
    double ring_radius;     /* R [m]; the grid must contain the ring with one node to spare */
    double mask_radius;     /* reconstruction mask radius [m], <= R (the paper uses 0.9 R) */
    double c0;              /* water sound speed [m/s] */
    double ds;              /* ray step [m] (Delta s of Def. ray-parameterisation) */
    int weight_mode;        /* 0: scattering-angle weight as printed (Eq. btk-amp-angle);
                               1: isochron weight |k_e + k_r| (App. D) */
    double tau;             /* step length of m <- m + tau dm (Sec. 3.4) */
    int precision;          /* rbx_precision of the two contractions */
} rbx_geometry;

typedef struct {
    double resid_norm2;     /* sum over r != e of |g_pred - data|^2 */
    double rms_dc;          /* RMS of the sound-speed change over the mask [m/s] */
    double max_abs_dc;      /* max |dc| over the mask [m/s] */
    double dm_norm;         /* ||dm||_2 over the mask [s^2/m^2] */
    long long n_uncovered;  /* (transducer, mask node) entries no ray triangle covered */
    long long n_clamped;    /* (e, r) pairs outside every exit-angle bracket */
    long long n_launches;   /* kernels launched by this call */
    float ms_trace;         /* smoothing, ray tracing and tables */
    float ms_forward;       /* direct Green's function, Born forward, residual */
    float ms_backproj;      /* back-projection and update */
    float ms_total;
    float ms_kernel[8];     /* per-kernel device time of the call: see RBX_K_* */
} rbx_stats;

/* indices into rbx_stats.ms_kernel */
#define RBX_K_TRACE 0       /* ray trace + ray-to-grid scatter */
#define RBX_K_SYNTH_FWD 1   /* Green's function synthesis for the forward; in an update on the
                               BF16 paths it also writes the back-projection's operands */
#define RBX_K_GEMM_FWD 2    /* Born forward contraction */
#define RBX_K_SYNTH_BP 3    /* reciprocal Green's function synthesis (about 0 where
                               RBX_K_SYNTH_FWD did it) */
#define RBX_K_GEMM_BP 4     /* back-projection contraction with fused row-dot */
#define RBX_K_FIELDS 5      /* smoothing + derivative fields */
#define RBX_K_TABLES 6      /* direct Green's function (+ angular density array, FP32) */
#define RBX_K_UPDATE 7      /* residual + update */

/* Create a job bound to a CUDA stream (a cudaStream_t; NULL means the legacy default
 * stream). All of the job's work is queued on that stream, so it is ordered with whatever
 * the caller queues there (e.g. the copies that fill its input buffers). The job starts
 * without geometry. */
rbx_status rbx_create(rbx_job **out, void *cuda_stream);

/* Set the grid, ring, transducer positions and options (Sec. 2.1, Sec. 6.3) and allocate the
 * job's device workspaces (tables of N x X entries, X = mask nodes). xducer_xy (host, 2N
 * doubles x_0, y_0, x_1, ...; copied) places transducer e at (x_e, y_e); NULL places them
 * uniformly, transducer e at R (cos 2 pi e/N, sin 2 pi e/N). Given positions must lie on the
 * ring (| |x_e| - R | <= 1e-6 R; the angle atan2(y_e, x_e) is kept) and run counterclockwise
 * around it once in index order, all distinct. Each transducer keeps the fan of N - 1 rays
 * at pi j / N from the tangent (Sec. 4.4 reading): the direct term interpolates between the
 * rays whose exits bracket each receiver, and receivers within about 2 pi / N of the emitter,
 * outside the fan's exit range, take the nearest ray (counted in rbx_stats.n_clamped); the
 * angular density is formed over the neighbouring indices e +/- 1.
 * Fails with RBX_EINVAL when the grid does not contain the ring, mask_radius > ring_radius,
 * N < 3, ds <= 0, a ray could need more than 2047 steps (2 R / ds), or the positions break
 * the rules above. Resets the model to water (c0). */
rbx_status rbx_set_geometry(rbx_job *job, const rbx_geometry *geom, const double *xducer_xy);

/* Number of mask nodes X and their row-major node indices (idx_dev: X int32, may be NULL). */
rbx_status rbx_mask(rbx_job *job, int *X_out, int *idx_dev);

/* Copy the sound-speed map c (ny*nx float32, m/s, device) into the job. RBX_ENUMERIC if
 * any value is not finite and positive (checked on the device, synchronises). */
rbx_status rbx_set_model(rbx_job *job, const float *c_dev);

/* Absorption and dispersion (Sec. 2.2, Szabo's power law): alpha0_dev is the absorption map
 * alpha0 [ny*nx] (float32, device, copied; Np (rad/s)^-y m^-1, alpha = alpha0 omega^y >= 0)
 * of the medium, known during the sound-speed inversion; y the power-law exponent (0 < y < 2,
 * y != 1). Rays then follow 1/c + alpha0 tan(pi y/2) omega^(y-1) (smoothed with the same
 * window as the lossless slowness), table amplitudes include exp(-int alpha ds), the Born
 * weights use Upsilon_m = omega c k~ and the update the lossy node factor (see
 * rbx_update_frequency). alpha0_dev == NULL returns the job to a lossless medium. Call after
 * rbx_set_geometry (which clears it); rays must be traced again afterwards.
 * Errors: RBX_EINVAL (bad y, negative or non-finite alpha0), RBX_ESTATE, RBX_ENOMEM. */
rbx_status rbx_set_absorption(rbx_job *job, const float *alpha0_dev, double y);

/* Integration mode (Sec. 6.3.2). mode 0 (default): travel times and amplitudes are integrated
 * on the smoothed map the rays follow, and the predicted data add the Born term of the rough
 * part m - m_s. mode 1, the paper's implementation: rays are still traced on the smoothed map,
 * but travel time, the amplitude's slowness ratio and absorption are integrated along them on
 * the non-smoothed maps, and the predicted data are the ray Green's functions alone (the
 * rough part is in their phase). Call after rbx_set_geometry (which resets it to 0); rays
 * must be traced again. Errors: RBX_EINVAL (mode not 0 or 1), RBX_ESTATE. */
rbx_status rbx_set_integration(rbx_job *job, int mode);

/* Ray linking of the direct term (Sec. 4.4, Sec. 6.3.2): max_rays > 0 links every emitter-
 * receiver pair by the secant method on the initial angle, started from the two fan rays whose
 * exits bracket the receiver and kept inside that bracket (regula falsi with the Illinois
 * weighting), until the exit lies within 1e-6 rad of it or max_rays new rays were traced; T and a are then interpolated in exit angle to the receiver exactly. The rays
 * follow the job's current smoothed map, integration mode and absorption. 0 (default): the
 * fan's exit-angle interpolation (one secant step's worth of accuracy). Applies to
 * rbx_direct_green, rbx_predict and every update. Pairs left unbracketed or unconverged are
 * counted in rbx_stats.n_clamped. Errors: RBX_EINVAL (max_rays < 0 or > 32), RBX_ESTATE. */
rbx_status rbx_set_linking(rbx_job *job, int max_rays);

/* One update from a set of nf frequencies (Sec. 6.3.2: the paper takes two consecutive
 * frequencies per update). The rays are traced once, on the map smoothed (and, when lossy,
 * dispersed) for freqs[0]; each frequency contributes its own residual and preconditioned
 * back-projection, and the search directions are summed before one step m <- m + tau dm.
 * data_dev: nf consecutive N x N complex64 blocks (device, emitter-major). nf == 1 is
 * rbx_update_frequency. out->resid_norm2 is summed over the set (no per-stage timings).
 * Synchronises. Errors: RBX_EINVAL (nf < 1 or > 16, bad frequencies), RBX_ESTATE, RBX_ENOMEM,
 * RBX_ENUMERIC as rbx_update_frequency. */
rbx_status rbx_update_set(rbx_job *job, const double *freqs_hz, int nf, double dfreq_hz, const void *data_dev,
                          rbx_stats *out);

/* Copy the job's current sound-speed map out (ny*nx float32, device). */
rbx_status rbx_get_model(rbx_job *job, float *c_dev);

/* Steps a1-a4 on the current model for frequency f: smooth the slowness with the
 * frequency's window (Sec. 6.2, 6.3.2), trace the ray fan of every transducer by Heun's
 * method with the paraxial system (Alg. 1), and scatter travel time, amplitude,
 * direction and caustic count onto the mask nodes (Sec. 4.4, Eqs. phase-discretised,
 * amplitude-geom-discretised); then the angular density |d gamma/d e| Delta e. */
rbx_status rbx_trace_rays(rbx_job *job, double freq_hz);

/* Replace the job's tables by caller-supplied ones ([N][X] device arrays: travel time
 * [s], reduced amplitude a [m^-1/2] (a = 0 marks an uncovered entry), direction angle
 * [rad], caustic count) and per-ray exit records exits_dev ([N][N-1][4] float32: exit
 * angle, T, a, K of ray j = 1..N-1). Used to run the contractions on given tables. */
rbx_status rbx_set_tables(rbx_job *job, const float *T_dev, const float *a_dev, const float *gamma_dev,
                          const uint8_t *K_dev, const float *exits_dev);

/* Copy the job's tables out (any pointer may be NULL): [N][X] arrays as in
 * rbx_set_tables plus dgamma ([N][X], |d gamma/d e| Delta e) and exits. */
rbx_status rbx_get_tables(rbx_job *job, float *T_dev, float *a_dev, float *gamma_dev, uint8_t *K_dev,
                          float *dgamma_dev, float *exits_dev);

/* Direct Green's function at the receivers from the ray fans (Eq. 2D_greens, step a5):
 * g[e*N + r] complex64, zero diagonal. */
rbx_status rbx_direct_green(rbx_job *job, double freq_hz, void *g_dev);

/* Ray-Born forward of a squared-slowness perturbation (Eqs. perturb1, derivative,
 * scattering-potential): D[e*N + r] = omega^2 dA sum_x G_r[x] G_e[x] dm[x] over the mask,
 * dm_dev ny*nx float32 [s^2/m^2]. Uses the tables of the last trace/set_tables. */
rbx_status rbx_forward(rbx_job *job, double freq_hz, const float *dm_dev, void *D_dev);

/* Predicted data on the current model: g_dir + F[m - m_s], m_s the smoothed squared
 * slowness of the tables' window (diagonal zero). Also the synthetic data generator. */
rbx_status rbx_predict(rbx_job *job, double freq_hz, void *g_dev);

/* Adjoint maps of a residual R (N x N complex64, device) onto the mask nodes
 * (out_dev: X complex64 in mask order).
 *  preconditioned = 0: F* R = omega^2 dA sum_{e,r} conj(G_r G_e) R[e,r] (Eq. functional-gradient, Q = 1).
 *  preconditioned = 1: sum_{e,r} W_er u_e u_r R[e,r], u_e = dgamma_e gdag_e (Eq. sound_speed_update2
 *  without its scalar factor Delta omega m / ((2 pi)^3 omega)). */
rbx_status rbx_adjoint(rbx_job *job, double freq_hz, const void *R_dev, void *out_dev, int preconditioned);

/* One Hessian-free update at frequency f with sweep spacing df (Delta omega = 2 pi df),
 * the update of Eqs. sound_speed_update / sound_speed_update2 with the step length of
 * Sec. 3.4: trace (a1-a4), direct Green's function, Born prediction and residual against
 * data_dev (N x N complex64, Eq. residual), preconditioned back-projection
 * dm = -(Delta omega / (2 pi)^3) (m / omega) Re sum_{e,r} W_er u_e u_r R[e,r], then
 * m <- m + tau dm on the mask and c = m^-1/2 (water outside the mask, Sec. 6.3).
 * Synchronises and fills *out (may be NULL). */
rbx_status rbx_update_frequency(rbx_job *job, double freq_hz, double dfreq_hz, const void *data_dev, rbx_stats *out);

/* Steps a5-a9 alone: one update on the job's current tables (from rbx_trace_rays or
 * rbx_set_tables) without re-tracing; the smoothed squared slowness m_s of the Born term is
 * recomputed from the current model with the window of freq_hz. */
rbx_status rbx_update_from_tables(rbx_job *job, double freq_hz, double dfreq_hz, const void *data_dev, rbx_stats *out);

/* As rbx_update_frequency with host buffers: copies data_host (N x N complex64; pinned
 * memory for an asynchronous copy) to the device on a copy stream of the job, beside the ray
 * trace, which does not read the data; runs the update and copies the updated model to
 * c_out_host (ny*nx float32, may be NULL), one wait for the model and the statistics. The
 * results are those of rbx_update_frequency, bit for bit. On RBX_ENUMERIC c_out_host holds
 * the model as kept (previous values at the failing nodes). */
rbx_status rbx_update_frequency_host(rbx_job *job, double freq_hz, double dfreq_hz, const void *data_host,
                                     float *c_out_host, rbx_stats *out);

/* Queue one update exactly as rbx_update_frequency does, without waiting for it: nothing is
 * copied to the host, so the call can be captured into a CUDA graph. Its scalar results go to
 * device stats slot `slot` (0..63) of the job; read them with rbx_get_stats. */
rbx_status rbx_update_frequency_async(rbx_job *job, double freq_hz, double dfreq_hz, const void *data_dev, int slot);

/* Wait for the job's stream and return the scalar results kept in stats slot `slot`
 * (timings are not filled). Returns the status the update in that slot ended with
 * (RBX_ENUMERIC, RBX_ETIMEOUT, ...). */
rbx_status rbx_get_stats(rbx_job *job, int slot, rbx_stats *out);

/* With on != 0, every later rbx_update_frequency_async records its stage events into the
 * events of its own stats slot (64 sets, created by this call), so rbx_get_stats also
 * returns that update's device timings (ms_trace, ms_forward, ms_backproj, ms_total,
 * ms_kernel) and its launch count, as rbx_update_frequency does. A slot's timings are those
 * of the last update queued into it. on == 0 frees the events (after waiting for the job's
 * stream). */
rbx_status rbx_set_slot_timing(rbx_job *job, int on);

/* Batched form: the full low-to-high sweeps of n independent jobs (slices of different
 * sizes), freqs[i][0..nf[i]-1] with data_dev[i] holding nf[i] N_i x N_i blocks, nf[i] <= 64.
 * Each job's sweep runs on a stream of its own, forked from and joined to one origin stream.
 * `use_graph` holds flags: with RBX_BATCH_GRAPH the whole fork/join is captured into one CUDA
 * graph and launched once, otherwise it is queued directly. With RBX_BATCH_GROUPED the jobs
 * go in lock-step by sweep step, and at each step one persistent launch traces the rays of
 * all the jobs still sweeping (a work list of (job, rays, fans) items that the GPU's blocks
 * take in turn, the jobs with the longest ray paths in the mask first); the rest of each
 * update stays on the job's stream. It needs the jobs to share their absorption and
 * integration settings, and is ignored otherwise. Without it, results are the same, bit for
 * bit, as running the jobs one after the other; with it, the grouped trace is a separate
 * compilation of the same arithmetic, whose tables agree with the per-job trace's to
 * rounding (the same coverage, travel times within 1e-10 s, amplitudes within 2e-5
 * relative but at near-caustic entries, where the amplitude is ill-conditioned, and the
 * caustic count of an entry at most rarely different), and it is deterministic itself. A
 * whole sweep carries that difference into the models as it carries the BF16 / FP32 one.
 * last[i] (nullable) receives job i's last update's scalars; ms_total (nullable) the device
 * time of the whole batch. The jobs' own streams are drained first and kept. */
#define RBX_BATCH_GRAPH 1
#define RBX_BATCH_GROUPED 2
rbx_status rbx_batch_run(rbx_job *const *jobs, int n, const double *const *freqs, const int *nf,
                         const void *const *data_dev, int use_graph, rbx_stats *last, float *ms_total);

/* Low-to-high frequency sweep (Sec. 3.4): one update per frequency freqs_hz[0..nf-1]
 * (host array), data_dev holding nf consecutive N x N complex64 blocks; df of frequency n
 * is half the distance between its neighbours (one-sided at the ends; 1 MHz / 10 when
 * nf == 1). per_freq (host, nf entries) may be NULL. */
rbx_status rbx_reconstruct(rbx_job *job, const double *freqs_hz, int nf, const void *data_dev, rbx_stats *per_freq);

/* Born forward for callers that cannot allocate device memory (inside a CUDA-graph capture
 * that must not add allocation nodes, under a framework allocator that owns the device, or
 * in services that forbid allocation after start-up). The paper has no counterpart: this is
 * a deployment variant of rbx_forward that needs no job. It computes
 * D[e*N + r] = sum_x G_r[x] G_e[x] v[x] from caller tables T_dev, a_dev (float32) and K_dev
 * (uint8), each [n_xducers][n_nodes] as in rbx_set_tables (a = 0: uncovered), and the Born
 * weights v_dev (n_nodes float32, v = omega^2 dA dm per mask node); D_dev is N x N complex64.
 * It allocates nothing: the split partial sums live in a fixed 8 MiB array inside the
 * library, so n_xducers must be <= 1024 (RBX_EINVAL otherwise). The contraction splits the
 * mask nodes over at most floor(2^20 / N^2) CTAs per tile pair (the array holds that many
 * N x N partial sums): at N = 1024 it runs unsplit, one CTA per upper 64 x 64 tile pair
 * (136 CTAs), each looping over all nodes, so the largest sizes run well below the speed of
 * rbx_forward. The first call on each
 * device looks up that array's device address (it may load the module): make it before any
 * stream capture. All calls share the array; calls that overlap on the GPU race and must be
 * serialised by the caller. Work is queued on cuda_stream (NULL: legacy default stream).
 * err (errlen bytes, may be NULL) receives a message, "" on success. */
rbx_status rbx_forward_noalloc(const float *T_dev, const float *a_dev, const uint8_t *K_dev, const float *v_dev,
                               int n_xducers, int n_nodes, double freq_hz, double c0, void *D_dev, void *cuda_stream,
                               char *err, size_t errlen);

/* ---------------------------------------------------------------- served form
 * A server takes reconstruction requests (host buffers) at any time and runs them with
 * continuous batching: a worker thread admits queued requests in arrival order while their
 * estimated device memory fits hbm_budget_bytes and fewer than max_inflight run; each runs its
 * whole low-to-high sweep (Sec. 3.4) on a stream of its own with data and model resident on
 * the device, overlapping the others; finished requests release their memory, which admits
 * the next. Results are the same as running each request alone. The server uses the CUDA
 * device current when it is created. */
typedef struct rbx_server rbx_server;

typedef enum {
    RBX_REQ_QUEUED = 0,
    RBX_REQ_RUNNING = 1,
    RBX_REQ_DONE = 2,
    RBX_REQ_FAILED = 3,
    RBX_REQ_CANCELLED = 4
} rbx_request_state;

rbx_status rbx_server_create(rbx_server **out, size_t hbm_budget_bytes, int max_inflight);

/* The server's admission estimate of the device bytes one request of this geometry and
 * nf frequencies reserves (an upper estimate of a job's workspaces plus its data). */
size_t rbx_estimate_bytes(const rbx_geometry *geom, int nf);

/* Queue a request: geometry, initial model c_init_host (ny*nx float32), frequencies
 * freqs_host[0..nf-1] (increasing, nf <= 64) and data_host (nf blocks of N x N complex64).
 * The inputs are copied; *ticket identifies the request. A request whose estimated memory
 * exceeds the budget fails with RBX_ENOMEM when it reaches the head of the queue. */
rbx_status rbx_server_submit(rbx_server *srv, const rbx_geometry *geom, const float *c_init_host,
                             const double *freqs_host, int nf, const void *data_host, long long *ticket);

/* State of a request (rbx_request_state). Once it has ended: latency_s = seconds from
 * submission to completion, and for a finished request c_out_host (ny*nx float32, nullable)
 * and last (nullable, scalars of its last update). Returns the request's final status once it
 * has ended (RBX_OK while it is queued or running). */
rbx_status rbx_server_poll(rbx_server *srv, long long ticket, int *state, double *latency_s, float *c_out_host,
                           rbx_stats *last);

/* Block until the request has ended or timeout_s passes (RBX_ETIMEOUT). */
rbx_status rbx_server_wait(rbx_server *srv, long long ticket, double timeout_s);

/* Cancel a request that is still queued (RBX_ESTATE once it runs). */
rbx_status rbx_server_cancel(rbx_server *srv, long long ticket);

/* Host-clock times of a request, in seconds since the server was created: submission,
 * admission (start of its device work; -1 while queued or if it never started) and end
 * (-1 while it has not ended). */
rbx_status rbx_server_times(rbx_server *srv, long long ticket, double *t_submit, double *t_start, double *t_end);

/* Requests queued and running, and the device bytes reserved by running ones. */
rbx_status rbx_server_info(rbx_server *srv, int *queued, int *running, size_t *bytes_in_use);

/* Error message of an ended request ("" if none); valid while the server exists. */
const char *rbx_server_error(rbx_server *srv, long long ticket);

/* Finish running requests, cancel queued ones, stop the worker and free the server. */
rbx_status rbx_server_destroy(rbx_server *srv);

/* Last error message of the job ("" if none). The string lives as long as the job. */
const char *rbx_last_error(const rbx_job *job);

/* Autotuning of the BF16 forward contraction's K split (split across CTAs of each upper
 * tile pair, partial sums reduced in a fixed order) and, on the plain BF16 path, of its
 * operand synthesis (separate pass or fused, see rbx_get_tuning_times). mode 1 (default): the
 * first job of a given (device, N, mask size, precision) in the process times up to five
 * split counts on its own operand planes inside rbx_set_geometry and keeps the fastest, then
 * the two syntheses at that split; later jobs of that shape reuse the choice, so results
 * within a process are reproducible. mode 0: the fixed
 * heuristic (about one CTA per SM), reproducible across processes. Other values only
 * query. Mode 2: the heuristic split with the fused-synthesis forward (see
 * rbx_get_tuning_times). Returns the previous mode. The choice changes the forward's
 * summation order, so results differ between split counts by rounding (within the BF16
 * tolerance). */
int rbx_autotune(int mode);

/* The forward K split the job uses and the number of candidates it timed (0: reused or
 * heuristic). */
rbx_status rbx_get_tuning(const rbx_job *job, int *fwd_splits, int *candidates_timed);

/* Diagnostic of the tuner's second choice on the plain BF16 path (the paper has no
 * counterpart): whether the Born forward forms its tensor-core operands from the tables inside
 * the contraction (fused synthesis of the Green's functions, Eq. 2D_greens) instead of reading
 * BF16 planes written by a separate synthesis pass. The tuner times, at the job's shape, the
 * separate pass over both contractions' operands plus the forward GEMM against the
 * back-projection's synthesis alone plus the fused forward, and keeps the faster. ms (4 floats,
 * nullable) receives those times in that order (0 where not timed); *fused (nullable) = 1 when
 * the job uses the fused forward. rbx_autotune(2) makes later jobs take the fused forward
 * without timing (heuristic split, plain BF16 only). */
rbx_status rbx_get_tuning_times(const rbx_job *job, float *ms, int *fused);

/* Device memory of the stream-ordered pool all jobs of the current device allocate from:
 * bytes held by live allocations (used) and bytes the pool has taken from the device
 * (reserved; freed workspaces stay reserved for reuse). trim != 0 first returns the unused
 * reserve to the device (after synchronising the device). Either pointer may be NULL. */
rbx_status rbx_pool_usage(size_t *used, size_t *reserved, int trim);

/* Diagnostic of the failure handling (the paper has no counterpart). Every wait of the
 * tensor-core kernels on a barrier or a copy is bounded: after one second of wall time
 * the kernel records a timeout, stops and frees what it holds, and the call returns
 * RBX_ETIMEOUT. This runs one kernel on the current device whose single thread waits, with
 * that same bound, on a barrier that nothing ever signals. *timed_out = 1 when the wait gave
 * up as it should (the expected result), 0 if the barrier completed. The call allocates and
 * frees 4 bytes of device memory, synchronises the device, takes about one second and leaves
 * the CUDA context usable. */
rbx_status rbx_selftest_bounded_wait(int *timed_out);

/* Wait for all work queued on the job's stream. */
rbx_status rbx_synchronize(rbx_job *job);

/* Wait for the job's stream, then free the job's device memory. */
rbx_status rbx_destroy(rbx_job *job);

#ifdef __cplusplus
}
#endif

#endif
