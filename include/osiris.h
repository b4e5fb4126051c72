/*
 * osiris.h -- C interface of the GB300 backward ray tracer for null geodesics
 * in Kerr space-time (Velasquez-Cadavid et al., "OSIRIS: A New Code for Ray
 * Tracing Around Compact Objects", arXiv:2202.00086).
 *
 * Conventions shared by every call
 *   - Geometrized units with the black-hole mass M = 1 (Sec. 1, last paragraph).
 *   - Boyer-Lindquist coordinates (t, r, theta, phi) and signature (-,+,+,+)
 *     (Sec. 4.3, Eq. Kerr).
 *   - One image-plane pixel = one backward null geodesic (Sec. 2.2). Pixel
 *     (i, j), 0 <= i < nx, 0 <= j < ny, sits at the cell centre
 *       x_i = x_min + (i + 1/2) (x_max - x_min) / nx,
 *       y_j = y_min + (j + 1/2) (y_max - y_min) / ny,
 *     and its outputs live at linear index j * nx + i.
 *   - Output arrays are caller-owned DEVICE pointers (any may be NULL when
 *     not wanted). The library never frees them.
 *   - Every launch is asynchronous on the caller's CUDA stream (a
 *     cudaStream_t passed as void*; NULL = the legacy default stream).
 *   - Return value 0 = OSIRIS_OK, negative = error (see osiris_strerror).
 *     Argument errors are detected on the host before anything is launched.
 *     No C++ exception crosses this interface.
 */
#ifndef OSIRIS_H
#define OSIRIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define OSIRIS_OK 0
#define OSIRIS_EINVAL (-1)   /* an argument is out of its documented range */
#define OSIRIS_ECUDA (-2)    /* a CUDA runtime call failed */
#define OSIRIS_ENOMEM (-3)   /* a caller-provided workspace is too small */
#define OSIRIS_ETIMEOUT (-4) /* a bounded wait ran out */

/* ---- per-ray status (the fate of the backward ray; Sec. 4.1, Sec. 5) ---- */
#define OSIRIS_STATUS_NONE 0     /* not traced */
#define OSIRIS_STATUS_CAPTURED 1 /* reached r < r_cap_factor * r_H */
#define OSIRIS_STATUS_ESCAPED 2  /* reached the celestial sphere r > r_esc_factor * r_obs */
#define OSIRIS_STATUS_DISK 3     /* hit the equatorial disk r_in <= r <= r_out */
#define OSIRIS_STATUS_MAXSTEP 4  /* step budget exhausted */
#define OSIRIS_STATUS_ERROR 5    /* state became non-finite */

/* ---- precision of the integrator -------------------------------------- */
#define OSIRIS_FP64 0  /* every operation in double precision */
#define OSIRIS_MIXED 1 /* stage evaluations of Hamilton's equations and the
                          sums over stages in FP32 around a double-float
                          state (each stage input is the state plus an FP32
                          increment); FP32 controller, end-point |H| in
                          double-float; for tolerances of 1e-8 and looser
                          (FP32 rounding of the stages swamps the error
                          estimate of tighter ones) */
#define OSIRIS_DF64 2  /* every operation of the integration in double-float
                          (pairs of FP32, 48-bit significand) on the FP32
                          pipe; FP64 for initial data and outputs */

/* ---- integrator (Sec. 3.1) -------------------------------------------- */
#define OSIRIS_RKCK45 0 /* Cash-Karp 4(5), six evaluations per attempt */
#define OSIRIS_RKDP45 1 /* Dormand-Prince 5(4), first same as last: six new
                           evaluations per attempt */

/* ---- space-times ------------------------------------------------------- */
#define OSIRIS_SPACETIME_KERR 0    /* Kerr, Boyer-Lindquist (Sec. 4.3), spin a */
#define OSIRIS_SPACETIME_QMETRIC 1 /* q-metric (Appendix A), quadrupole q, m = 1 */

/* ---- counters written to osiris_trace_opts.stats (uint64 each) --------- */
#define OSIRIS_STAT_RAYS 0          /* rays finished */
#define OSIRIS_STAT_ACCEPTED 1      /* accepted Cash-Karp steps */
#define OSIRIS_STAT_REJECTED 2      /* rejected Cash-Karp steps */
#define OSIRIS_STAT_ROOT_STEPS 3    /* steps spent locating stopping surfaces */
#define OSIRIS_STAT_RHS_EVALS 4     /* evaluations of Hamilton's equations */
#define OSIRIS_STAT_STATUS0 5       /* 5..10: rays per status code 0..5 */
#define OSIRIS_STAT_MAX_ABS_H 11    /* max |H| over all rays that did not end in
                                       OSIRIS_STATUS_ERROR, as IEEE-754 bits */
#define OSIRIS_STAT_FP64_STEPS 12   /* attempts taken in FP64: every attempt of
                                       the FP64 kernels, none in MIXED or DF64 */
#define OSIRIS_STAT_CHECK_FAILS 13  /* bounds-checked build only: failed index checks */
#define OSIRIS_STAT_CHECK_WORST 14  /* bounds-checked build only: max over failures of
                                       (check code << 56) | ray index; codes 1 ray index
                                       outside the launch, 2 request index, 3 ray outside
                                       its request's range, 4 pixel / state index */
#define OSIRIS_STATS_LEN 16

/* Opaque camera: space-time, observer and image plane. Host memory only. */
typedef struct osiris_camera osiris_camera;

/* Integration options. Fill with osiris_default_opts, then override. */
typedef struct {
    double tol;            /* per-step tolerance of the embedded error estimate
                              (error norm: max over r, theta, phi, p_r, p_theta of
                              |y5 - y4| / (tol (1 + max(|y_n|, |y_n+1|)))), > 0 */
    int64_t max_steps;     /* cap on accepted + rejected steps per ray, >= 1 */
    int32_t precision;     /* OSIRIS_FP64, OSIRIS_MIXED or OSIRIS_DF64 */
    int32_t persistent;    /* 0: one ray per thread; 1: persistent grid that
                              refills lanes from a device ray queue (needs
                              workspace) */
    double r_cap_factor;   /* captured when r < r_cap_factor * r_H, > 1 */
    double r_esc_factor;   /* escaped when r > r_esc_factor * r_obs, > 1 */
    double cell_deg;       /* celestial checkerboard cell, degrees, (0, 180] */
    double cell_phase_deg; /* longitude offset of the checkerboard, degrees */
    int32_t block_size;    /* threads per block, multiple of 32 in [32, 256];
                              0 = library default */
    int32_t blocks_per_sm; /* persistent grid: blocks per SM; 0 = occupancy limit */
    uint64_t* stats;       /* optional DEVICE array of OSIRIS_STATS_LEN counters;
                              the call adds to them (zero it first) */
    void* workspace;       /* DEVICE scratch, >= osiris_workspace_bytes(n) bytes,
                              256-byte aligned; required when persistent != 0 or
                              for osiris_trace_batch. Not shared between calls
                              that may run at the same time. */
    size_t workspace_bytes;
    int32_t integrator;    /* OSIRIS_RKCK45 (default) or OSIRIS_RKDP45 */
    int32_t rays_per_lane; /* rays a lane takes at once, 0..64 (0 = 1): a plain
                              launch gives each thread this many consecutive
                              pixels; a persistent grid claims this many per
                              idle lane with each queue atomic */
    int32_t refill_lanes;  /* persistent grid, 0..32 (0 = library default: 4,
                              32 in OSIRIS_MIXED): a
                              warp whose other lanes are still integrating
                              refills its idle lanes only once at least this
                              many are idle (a warp with no busy lane always
                              refills) */
} osiris_trace_opts;

/* Per-ray outputs: DEVICE arrays with one entry per ray (NULL = not wanted).
 * Shadow/lensing outputs (Sec. 3.2, Sec. 4):
 *   status      fate (OSIRIS_STATUS_*)
 *   r,theta,phi final Boyer-Lindquist position; on the stopping surface for
 *               CAPTURED / ESCAPED / DISK; theta and phi are not wrapped
 *   max_abs_H   max |H| over the initial point, every accepted point and the
 *               final point (Sec. 3.1, Error = |H_num|)
 *   steps       accepted Cash-Karp steps
 *   cell_i/j    ESCAPED: checkerboard cell (theta folded into [0, pi], phi
 *               wrapped into [0, 2pi) after adding the phase); else -1
 *   parity      ESCAPED: (cell_i + cell_j) mod 2; else 0
 * Disk outputs (Sec. 5), DISK rays only (0 elsewhere):
 *   g           redshift nu_obs / nu_em, nu_obs = 1 in the observer's frame
 *   intensity   g^3 r_hit^-2
 *   r_hit       radius of the first crossing inside [r_in, r_out] */
typedef struct {
    uint8_t* status;
    double* r;
    double* theta;
    double* phi;
    double* max_abs_H;
    uint32_t* steps;
    int16_t* cell_i;
    int16_t* cell_j;
    uint8_t* parity;
    double* g;
    double* intensity;
    double* r_hit;
} osiris_outputs;

/* Sets the defaults: tol 1e-10, max_steps 1e6, FP64, Cash-Karp,
 * non-persistent, r_cap_factor 1.01, r_esc_factor 1.1, 10-degree cells,
 * phase 0, library block size, no stats, no workspace, library work
 * distribution (one ray per lane at a time, refill once four lanes of a warp
 * are idle). */
void osiris_default_opts(osiris_trace_opts* opts);

/* Create a camera (Sec. 2.3, Eq. momentums; observer at t0 = 0, phi0 = 0):
 *   a          spin, 0 <= a < 1
 *   r_obs      observer radius, > 10 r_H
 *   incl_deg   observer polar angle theta0 in degrees, (0, 180)
 *   x/y_min/max image-plane extent (x_min < x_max, y_min < y_max); every
 *              corner must satisfy x^2 + y^2 < r_obs^2
 *   nx, ny     resolution, >= 1 each
 * The observer is a zero angular momentum observer; a pixel (x, y) gets
 *   p_theta = y sqrt(g_thth)/r_obs, L = p_phi = -x sqrt(g_phph)/r_obs,
 *   E = -p_t = 1/A_t + x g_tphi/(r_obs sqrt(g_phph)),
 *   p_r = -sqrt(g_rr (1 - (x^2 + y^2)/r_obs^2)),
 * with A_t = sqrt(g_phph / (g_tphi^2 - g_tt g_phph)) and the metric at
 * (r_obs, theta0). Host-only: no device work, no allocation on the device.
 * On success *out owns host memory released by osiris_destroy_camera. */
int osiris_init_camera(osiris_camera** out, double a, double r_obs, double incl_deg,
                       double x_min, double x_max, double y_min, double y_max, int32_t nx,
                       int32_t ny);

/* Camera in the q-metric (Appendix A, Eq. q-metric with m = 1, written in
 * signature (-,+,+,+)): g_tt = -f^(1+q), g_rr = f^(-1-q) X^-k,
 * g_thth = f^-q r^2 X^-k, g_phph = f^-q r^2 sin^2, f = 1 - 2/r,
 * X = 1 + sin^2/(r^2 - 2r), k = q (2 + q). q = 0 is Schwarzschild; q in
 * (-1, -1 + sqrt(3/2)) \ {0} describes naked singularities. The initial data
 * are those of osiris_init_camera for this static metric; rays end at
 * r < r_cap_factor * 2 (the singular surface r = 2) or at the celestial
 * sphere. q-metric renders run in every precision, without a disk.
 *   q          > -1; r_obs > 20; the other arguments as osiris_init_camera. */
int osiris_init_camera_q(osiris_camera** out, double q, double r_obs, double incl_deg,
                         double x_min, double x_max, double y_min, double y_max, int32_t nx,
                         int32_t ny);

void osiris_destroy_camera(osiris_camera* cam);

/* Number of rays (nx * ny) of a camera. */
int64_t osiris_camera_rays(const osiris_camera* cam);

/* Shadow and lensing render (Sec. 3.2, Sec. 4): trace every pixel of the
 * camera until capture, escape, the step cap or a non-finite state. Rays are
 * integrated with Hamilton's equations (Sec. 2.1) by adaptive Cash-Karp 4(5)
 * steps (Sec. 3.1); the capture and escape surfaces are located inside the
 * last step. Outputs hold osiris_camera_rays(cam) entries. */
int osiris_trace(const osiris_camera* cam, const osiris_trace_opts* opts,
                 const osiris_outputs* out, void* cuda_stream);

/* Thin-disk render (Sec. 5): as osiris_trace, and a ray also stops at its
 * first crossing of the equatorial plane with r_in <= r <= r_out, where a
 * Keplerian disk (Omega = 1 / (r^3/2 + a)) gives the redshift g and the
 * intensity g^3 r^-2. Requires r_cap_factor * r_H < r_in < r_out < r_esc. */
int osiris_render_disk(const osiris_camera* cam, double r_in, double r_out,
                       const osiris_trace_opts* opts, const osiris_outputs* out,
                       void* cuda_stream);

/* Disk models (Sec. 5): how the gas on circular equatorial orbits moves. */
#define OSIRIS_DISK_NONE 0      /* shadow / lensing render */
#define OSIRIS_DISK_KEPLERIAN 1 /* Omega = 1 / (r^3/2 + a) */
#define OSIRIS_DISK_CONSTANT_L 2 /* constant specific angular momentum
                                    l0 = -u_phi / u_t:
                                    Omega = -(g_tphi + l0 g_tt) / (g_phph + l0 g_tphi) */

/* Thin-disk render with a disk of constant specific angular momentum l0
 * (Sec. 5): as osiris_render_disk, with Omega = -(g_tphi + l0 g_tt) /
 * (g_phph + l0 g_tphi) at the hit radius. Where that motion is not timelike
 * (g_ab u^a u^b = -1 has no solution) the hit still stops the ray and g and
 * the intensity are 0. l0 must be finite. */
int osiris_render_disk_l0(const osiris_camera* cam, double r_in, double r_out, double l0,
                          const osiris_trace_opts* opts, const osiris_outputs* out,
                          void* cuda_stream);

/* One render (or one contiguous range of its pixels) of a batch. */
typedef struct {
    const osiris_camera* camera;
    int32_t disk;        /* OSIRIS_DISK_NONE, _KEPLERIAN or _CONSTANT_L */
    double r_in, r_out;  /* disk radii (disk = 1) */
    double tol;          /* per-request tolerance; <= 0 takes opts->tol */
    osiris_outputs out;  /* DEVICE outputs of the whole render (nx * ny entries) */
    int64_t first_ray;   /* first pixel index traced by this entry */
    int64_t n_rays;      /* pixels [first_ray, first_ray + n_rays) are traced and their
                            outputs written; n_rays <= 0 means the whole render
                            (first_ray must then be 0). A range must lie inside
                            [0, nx * ny). */
    double l0;           /* specific angular momentum (disk = OSIRIS_DISK_CONSTANT_L) */
} osiris_request;

/* Bytes of DEVICE workspace that osiris_trace_batch needs for n requests
 * (also enough for osiris_trace / osiris_render_disk with persistent = 1
 * when n = 1). */
size_t osiris_workspace_bytes(int32_t n_requests);

/* Batched uneven renders in ONE persistent launch: the rays of all requests
 * form one device queue; lanes that finish a ray take the next one, whatever
 * its request. Each request's outputs are those of the corresponding single
 * call. opts->workspace must hold osiris_workspace_bytes(n) bytes; the
 * request table is copied into it on the stream (the host array may be
 * reused when the call returns). 1 <= n_requests <= 65536. */
int osiris_trace_batch(const osiris_request* reqs, int32_t n_requests,
                       const osiris_trace_opts* opts, void* cuda_stream);

/* Batch plan: a batched persistent launch (osiris_trace_batch) recorded once
 * as a CUDA graph and replayed per batch, for request loops that launch many
 * rounds (the continuous-batching server). The graph holds the upload of the
 * request table from a pinned host staging table (all max_requests entries),
 * the reset of the device ray queue and the trace kernel; each launch
 * rewrites the staging table and patches the kernel arguments and the grid
 * into the instantiated graph, then launches it: one API launch per round.
 * Results are those of osiris_trace_batch with the same requests and opts. */
typedef struct osiris_batch_plan osiris_batch_plan;

/* Create a plan for batches of up to max_requests (1..65536) requests in the
 * given space-time (OSIRIS_SPACETIME_*), with opts fixed for the plan's life:
 * precision, integrator, launch shape, stats and per-request defaults
 * (tol <= 0 in a request takes opts->tol). opts->workspace (DEVICE, >=
 * osiris_workspace_bytes(max_requests) bytes) belongs to the plan until it is
 * destroyed and must not be used by other calls meanwhile. The plan allocates
 * max_requests table entries of pinned host memory. Returns OSIRIS_EINVAL
 * (bad arguments), OSIRIS_ENOMEM (workspace too small
 * or no pinned memory) or OSIRIS_ECUDA; *plan is NULL on error. */
int osiris_batch_plan_create(osiris_batch_plan** plan, int32_t max_requests, int32_t spacetime,
                             const osiris_trace_opts* opts);

/* Launch one batch (1 <= n_requests <= max_requests, all in the plan's
 * space-time) on cuda_stream, asynchronously. Requests are validated as in
 * osiris_trace_batch; the host array may be reused when the call returns.
 * Before rewriting the staging table the call waits (host) until the
 * previous launch of this plan has uploaded it. Launches of one plan must be
 * ordered (one stream, or streams the caller orders), since they share the
 * device table and queue; use one plan per batch in flight. Not thread-safe
 * per plan. */
int osiris_batch_plan_launch(osiris_batch_plan* plan, const osiris_request* reqs,
                             int32_t n_requests, void* cuda_stream);

/* Free a plan (NULL is ignored). Waits for the last upload; launches already
 * queued still complete. */
void osiris_batch_plan_destroy(osiris_batch_plan* plan);

/* Most requests osiris_trace_batch_static takes in one call. */
#define OSIRIS_STATIC_MAX_REQUESTS 256

/* Allocation-free variant of osiris_trace_batch. The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory themselves, e.g. a plug-in inside a host application that
 * owns every device allocation, a process running under a device-memory
 * quota where a fresh allocation may fail at a bad moment, or a render loop
 * that must not call cudaMalloc/cudaFree because those calls can synchronize
 * the whole device.
 * Instead of opts->workspace (ignored here, as is opts->workspace_bytes), the
 * queue counter and request table live in a fixed array in device memory
 * that the library reserves when it is loaded on a device: 256 bytes plus
 * room for OSIRIS_STATIC_MAX_REQUESTS requests (about 90 KB). Every GPU that
 * loads the library holds that array until the process exits. The caller
 * still owns the cameras and every output array, as with osiris_trace_batch,
 * and the outputs are the same.
 *   - n_requests must be in [1, OSIRIS_STATIC_MAX_REQUESTS]; more returns
 *     OSIRIS_EINVAL before anything is launched.
 *   - The first call on a device looks up the device address of the array
 *     (once per device, with that device current).
 *   - All calls share the one array, which keeps the last call's contents;
 *     each call resets the queue counter and rewrites the request table on
 *     its stream. Calls whose work may overlap on the GPU (different streams
 *     without ordering between them) race on the array: serialize them.
 *   - No cudaMalloc, cudaFree or other allocating routine is called. */
int osiris_trace_batch_static(const osiris_request* reqs, int32_t n_requests,
                              const osiris_trace_opts* opts, void* cuda_stream);

/* Test hook: trace n rays from explicit initial data instead of pixels.
 * states: DEVICE array of n rows (t, r, theta, phi, p_r, p_theta) (t unused);
 * E, L: DEVICE arrays of n constants (p_t = -E, p_phi = L). r_obs sets the
 * escape radius. disk = 1 adds the disk of osiris_render_disk. Outputs hold
 * n entries. */
int osiris_trace_states(double a, double r_obs, const double* states, const double* E,
                        const double* L, int64_t n, int32_t disk, double r_in, double r_out,
                        const osiris_trace_opts* opts, const osiris_outputs* out,
                        void* cuda_stream);

/* Test hook for either space-time and for massive particles: as
 * osiris_trace_states, with spacetime = OSIRIS_SPACETIME_KERR (param = a) or
 * OSIRIS_SPACETIME_QMETRIC (param = q), and mass2 = 0 for light (H = 0) or
 * 1 for a unit-mass particle on the shell H = -1/2 (time-like geodesics,
 * Sec. 2.1 and Appendix A). max_abs_H then reports max |H - H_shell|. The
 * q-metric needs OSIRIS_FP64 or OSIRIS_DF64, and disk = 0. */
int osiris_trace_states_ex(int32_t spacetime, double param, double r_obs, double mass2,
                           const double* states, const double* E, const double* L, int64_t n,
                           int32_t disk, double r_in, double r_out, const osiris_trace_opts* opts,
                           const osiris_outputs* out, void* cuda_stream);

/* Copy n entries of every non-NULL field of dev (DEVICE) to the same field of
 * host (HOST, preferably pinned), asynchronously on the stream. Fields that
 * are NULL in either struct are skipped. */
int osiris_copy_outputs_to_host(const osiris_outputs* dev, const osiris_outputs* host,
                                int64_t n, void* cuda_stream);

/* Prograde ISCO radius (Bardeen, Press & Teukolsky 1972) for the disk inner
 * edge r_in = r_isco(a) (Sec. 5 uses r_in = r_isco). Host-only. */
double osiris_isco(double a);

/* Horizon radius r_H = 1 + sqrt(1 - a^2) (Sec. 4.3). Host-only. */
double osiris_horizon(double a);

/* Throughput probes for the roofline denominators (the trace kernels are
 * bound by the FP64 pipe, and the double-float kernels by the FP32 pipe; the
 * paper has no counterpart). osiris_pipe_probe launches one kernel of
 * n_threads threads (256 per block), each running 16 independent chains of
 * `iters` x 4 operations of one kind:
 *   op 0  fused multiply-add a = a b + c (2 floating-point operations)
 *   op 1  multiply a = a b (1)
 *   op 2  add a = a + c (1)
 *   op 3  the multiply written as a fused multiply-add with a zero addend (1)
 *   op 4  the add written as a fused multiply-add by one (1)
 * in FP64 (precision = OSIRIS_FP64) or FP32 (OSIRIS_MIXED), and stores one
 * value per thread in dev_out (DEVICE, n_threads doubles). *flops receives
 * the floating-point operations of the launch. n_threads must be a positive
 * multiple of 256; osiris_pipe_probe_threads gives the count that fills
 * every SM of the current device with resident blocks (SMs x resident
 * blocks x 256), or a negative error code. Time the launch with events on
 * the stream. */
int osiris_pipe_probe(int32_t precision, int32_t op, int64_t n_threads, int32_t iters,
                      double* dev_out, double* flops, void* cuda_stream);
int64_t osiris_pipe_probe_threads(int32_t precision, int32_t op);

/* osiris_pipe_probe with op 0 (fused multiply-add). */
int osiris_fma_probe(int32_t precision, int64_t n_threads, int32_t iters, double* dev_out,
                     double* flops, void* cuda_stream);

/* Bounded host wait for the work queued on a stream (the calls above are
 * asynchronous): polls the stream until it is idle or timeout_s seconds
 * (>= 0, finite) have passed. Returns OSIRIS_OK when the work is complete,
 * OSIRIS_ETIMEOUT when the bound ran out first (the work stays queued and
 * the call may be repeated), OSIRIS_ECUDA when the stream reports an error,
 * OSIRIS_EINVAL for a negative or non-finite bound. Polls every ~50 us. The
 * paper has no counterpart: it exists so that a request loop never blocks
 * without a bound. */
int osiris_stream_wait(void* cuda_stream, double timeout_s);

/* Human-readable text for a return code. */
const char* osiris_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* OSIRIS_H */
