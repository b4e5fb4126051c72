// Host side of the C interface declared in include/osiris.h: argument
// validation, the per-camera constants of the initial data (Sec. 2.3), and
// the launches. No allocation happens here: outputs and workspace belong to
// the caller.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <thread>
#include <new>
#include <vector>

#include "osiris_internal.h"

using osiris_impl::Kernel;
using osiris_impl::KernelArgs;
using osiris_impl::ReqDev;

struct osiris_camera {
  int32_t spacetime;  // OSIRIS_SPACETIME_*
  double q;           // q-metric quadrupole
  double a, r0, incl_deg, th0;
  double x_min, x_max, y_min, y_max;
  int32_t nx, ny;
  // observer terms of the initial momenta
  double inv_At, e_x, l_x, pth_y, grr;
};

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kDefaultBlock = 128;

bool is_fin(double v) { return std::isfinite(v); }

double horizon(double a) { return 1.0 + std::sqrt(1.0 - a * a); }

// Inner stopping surface scale: Kerr horizon, or the q-metric's r = 2.
double inner_radius(int spacetime, double a) {
  return spacetime == OSIRIS_SPACETIME_QMETRIC ? 2.0 : horizon(a);
}

int check_opts(const osiris_trace_opts* o) {
  if (!o) return OSIRIS_EINVAL;
  if (!(o->tol > 0.0) || !is_fin(o->tol)) return OSIRIS_EINVAL;
  if (o->max_steps < 1) return OSIRIS_EINVAL;
  if (o->precision != OSIRIS_FP64 && o->precision != OSIRIS_MIXED && o->precision != OSIRIS_DF64)
    return OSIRIS_EINVAL;
  if (o->integrator != OSIRIS_RKCK45 && o->integrator != OSIRIS_RKDP45) return OSIRIS_EINVAL;
  if (!(o->r_cap_factor > 1.0) || !is_fin(o->r_cap_factor)) return OSIRIS_EINVAL;
  if (!(o->r_esc_factor > 1.0) || !is_fin(o->r_esc_factor)) return OSIRIS_EINVAL;
  if (!(o->cell_deg > 0.0 && o->cell_deg <= 180.0)) return OSIRIS_EINVAL;
  if (!is_fin(o->cell_phase_deg)) return OSIRIS_EINVAL;
  if (o->block_size != 0 &&
      (o->block_size < 32 || o->block_size > 256 || o->block_size % 32 != 0))
    return OSIRIS_EINVAL;
  if (o->blocks_per_sm < 0) return OSIRIS_EINVAL;
  if (o->rays_per_lane < 0 || o->rays_per_lane > 64) return OSIRIS_EINVAL;
  if (o->refill_lanes < 0 || o->refill_lanes > 32) return OSIRIS_EINVAL;
  if (o->workspace && (reinterpret_cast<uintptr_t>(o->workspace) & 255u)) return OSIRIS_EINVAL;
  return OSIRIS_OK;
}

int check_disk(double a, double r_cap_factor, double r_esc, double r_in, double r_out) {
  if (!is_fin(r_in) || !is_fin(r_out)) return OSIRIS_EINVAL;
  if (!(r_in > r_cap_factor * horizon(a))) return OSIRIS_EINVAL;
  if (!(r_in < r_out) || !(r_out < r_esc)) return OSIRIS_EINVAL;
  return OSIRIS_OK;
}

// Fields common to pixel and explicit-state requests.
void fill_common(ReqDev& R, double a, double r0, const osiris_trace_opts* o, double tol,
                 int disk, double r_in, double r_out, const osiris_outputs* out,
                 double l0 = 0.0, int spacetime = OSIRIS_SPACETIME_KERR, double q = 0.0,
                 double mass2 = 0.0) {
  R.spacetime = spacetime;
  R.a = a;
  R.q = q;
  R.H0 = -0.5 * mass2;
  R.r0 = r0;
  R.r_cap = o->r_cap_factor * inner_radius(spacetime, a);
  R.r_esc = o->r_esc_factor * r0;
  R.disk = disk;
  R.r_in = disk ? r_in : 0.0;
  R.r_out = disk ? r_out : 0.0;
  R.l0 = disk == OSIRIS_DISK_CONSTANT_L ? l0 : 0.0;
  R.tol = tol > 0.0 ? tol : o->tol;
  R.h0 = 0.01 * r0;
  R.max_steps = o->max_steps;
  R.cell_rad = o->cell_deg * kPi / 180.0;
  R.inv_cell = 1.0 / R.cell_rad;
  R.phase_rad = o->cell_phase_deg * kPi / 180.0;
  R.n_th_cells = static_cast<int32_t>(std::ceil(180.0 / o->cell_deg - 1e-9));
  R.n_ph_cells = static_cast<int32_t>(std::ceil(360.0 / o->cell_deg - 1e-9));
  R.out = *out;
}

void fill_camera(ReqDev& R, const osiris_camera* c) {
  R.th0 = c->th0;
  R.x_min = c->x_min;
  R.x_span = c->x_max - c->x_min;
  R.y_min = c->y_min;
  R.y_span = c->y_max - c->y_min;
  R.nx = c->nx;
  R.ny = c->ny;
  R.inv_At = c->inv_At;
  R.e_x = c->e_x;
  R.l_x = c->l_x;
  R.pth_y = c->pth_y;
  R.grr = c->grr;
  R.explicit_states = 0;
  R.states = R.E = R.L = nullptr;
  R.n_rays = static_cast<int64_t>(c->nx) * c->ny;
  R.pixel_offset = 0;
}

// Pixel range of a batch entry (the whole render when n_rays <= 0).
int apply_range(ReqDev& R, const osiris_request& q) {
  if (q.n_rays <= 0) return q.first_ray == 0 ? OSIRIS_OK : OSIRIS_EINVAL;
  if (q.first_ray < 0 || q.first_ray > R.n_rays || q.n_rays > R.n_rays - q.first_ray)
    return OSIRIS_EINVAL;
  R.pixel_offset = q.first_ray;
  R.n_rays = q.n_rays;
  return OSIRIS_OK;
}

int cuda_rc(int e) { return e == 0 ? OSIRIS_OK : OSIRIS_ECUDA; }

// Every precision traces both space-times; the q-metric has no disk model.
int check_spacetime(int spacetime, int disk) {
  if (spacetime == OSIRIS_SPACETIME_KERR) return OSIRIS_OK;
  if (spacetime != OSIRIS_SPACETIME_QMETRIC) return OSIRIS_EINVAL;
  if (disk) return OSIRIS_EINVAL;
  return OSIRIS_OK;
}

int sm_count(int* n) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OSIRIS_ECUDA;
  if (cudaDeviceGetAttribute(n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return OSIRIS_ECUDA;
  return OSIRIS_OK;
}

using Launcher = int (*)(const KernelArgs&, Kernel, int, int, int, void*);

Launcher launcher_of(const osiris_trace_opts* o) {
  return (o->precision == OSIRIS_MIXED)  ? osiris_impl::launch_trace_mixed
         : (o->precision == OSIRIS_DF64) ? osiris_impl::launch_trace_df64
                                         : osiris_impl::launch_trace_fp64;
}

// Launch shape of a persistent grid: threads per block and the full grid
// (SMs x resident blocks per SM of the kernel that will run).
int persistent_shape(const osiris_trace_opts* o, int spacetime, int* block,
                     int64_t* full_grid) {
  *block = o->block_size ? o->block_size : kDefaultBlock;
  int sms = 0;
  if (int rc = sm_count(&sms)) return rc;
  int per_sm = o->blocks_per_sm;
  if (per_sm == 0) {
    auto occ = (o->precision == OSIRIS_MIXED)  ? osiris_impl::occupancy_mixed
               : (o->precision == OSIRIS_DF64) ? osiris_impl::occupancy_df64
                                               : osiris_impl::occupancy_fp64;
    if (occ(Kernel::kPersistent, o->integrator, spacetime, *block, &per_sm) != 0 || per_sm < 1)
      return OSIRIS_ECUDA;
  }
  *full_grid = static_cast<int64_t>(sms) * per_sm;
  return OSIRIS_OK;
}

// Work-distribution knobs of a launch (0 in the options = the library
// default: one ray per lane; refill once 4 lanes of a busy warp are idle, or
// in MIXED once all 32 are). Measured on the 12 x 1024^2 Kerr set, refill
// granularity 1 / 4 / 8 / 16 / 32: DF64 16.2 / 18.5-19.0 / 18.1 / 18.5 / 18.9
// Mrays/s, FP64 3.59 / 3.79 / 3.69 / 3.70 / 3.75; MIXED at tol 1e-8 49.0 /
// 65.3 / 65.5 / 67.5 / 70.2 (double-float stepper), refill 4 / 8 / 16 / 32:
// 94.7 / 96.7 / 100.7 / 106.1 (FP32 stage sums, rolled), 16 / 32: 148.5 /
// 162.2 (the current stepper). A MIXED ray takes about half
// the attempts of a DF64 ray at tol 1e-10, so its start and end (FP64 work,
// one warp instruction however many lanes share it) weigh more, and starting
// a warp's rays together also keeps neighbouring pixels in one warp.
constexpr int kDefaultRaysPerLane = 1;
constexpr int kDefaultRefillLanes = 4;
constexpr int kDefaultRefillLanesMixed = 32;

void set_granularity(KernelArgs& args, const osiris_trace_opts* o) {
  args.rays_per_lane = o->rays_per_lane > 0 ? o->rays_per_lane : kDefaultRaysPerLane;
  args.refill_lanes = o->refill_lanes > 0 ? o->refill_lanes
                      : o->precision == OSIRIS_MIXED ? kDefaultRefillLanesMixed
                                                     : kDefaultRefillLanes;
}

// Launch the trace kernel for the requests in args (args.reqs / single).
int launch(KernelArgs& args, const osiris_trace_opts* o, void* stream) {
  if (args.total_rays == 0) return OSIRIS_OK;
  const bool persistent = o->persistent != 0 || args.reqs != nullptr;
  const Launcher launcher = launcher_of(o);
  set_granularity(args, o);
  if (!persistent) {
    const int block = o->block_size ? o->block_size : kDefaultBlock;
    const int64_t per_block = static_cast<int64_t>(block) * args.rays_per_lane;
    const int64_t grid = (args.total_rays + per_block - 1) / per_block;
    if (grid > 0x7fffffff) return OSIRIS_EINVAL;
    args.queue = nullptr;
    return cuda_rc(
        launcher(args, Kernel::kPlain, o->integrator, static_cast<int>(grid), block, stream));
  }
  if (!o->workspace || o->workspace_bytes < osiris_impl::kQueueBytes) return OSIRIS_ENOMEM;
  int block = 0;
  int64_t grid = 0;
  const int spacetime = args.reqs ? args.spacetime : args.single.spacetime;
  if (int rc = persistent_shape(o, spacetime, &block, &grid)) return rc;
  const int64_t per_block = static_cast<int64_t>(block) * args.rays_per_lane;
  const int64_t needed = (args.total_rays + per_block - 1) / per_block;
  if (grid > needed) grid = needed;
  args.queue = static_cast<unsigned long long*>(o->workspace);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(args.queue, 0, sizeof(unsigned long long), s) != cudaSuccess)
    return OSIRIS_ECUDA;
  return cuda_rc(
      launcher(args, Kernel::kPersistent, o->integrator, static_cast<int>(grid), block, stream));
}

// Validate a batch and fill its request table (host memory, n entries);
// *total receives the number of rays. All requests share one space-time.
int build_table(const osiris_request* reqs, int32_t n, const osiris_trace_opts* o,
                ReqDev* table, int64_t* total) {
  int64_t begin = 0;
  for (int32_t k = 0; k < n; ++k) {
    const osiris_request& q = reqs[k];
    if (!q.camera) return OSIRIS_EINVAL;
    if (q.tol < 0.0 || !is_fin(q.tol)) return OSIRIS_EINVAL;
    if (q.disk < OSIRIS_DISK_NONE || q.disk > OSIRIS_DISK_CONSTANT_L || !is_fin(q.l0))
      return OSIRIS_EINVAL;
    if (q.camera->spacetime != reqs[0].camera->spacetime) return OSIRIS_EINVAL;
    if (int rc = check_spacetime(q.camera->spacetime, q.disk)) return rc;
    const double r_esc = o->r_esc_factor * q.camera->r0;
    if (q.disk)
      if (int rc = check_disk(q.camera->a, o->r_cap_factor, r_esc, q.r_in, q.r_out)) return rc;
    ReqDev& R = table[k];
    std::memset(&R, 0, sizeof(R));
    fill_common(R, q.camera->a, q.camera->r0, o, q.tol, q.disk, q.r_in, q.r_out, &q.out, q.l0,
                q.camera->spacetime, q.camera->q);
    fill_camera(R, q.camera);
    if (int rc = apply_range(R, q)) return rc;
    R.ray_begin = begin;
    begin += R.n_rays;
  }
  *total = begin;
  return OSIRIS_OK;
}

int run_camera(const osiris_camera* cam, int disk, double r_in, double r_out, double l0,
               const osiris_trace_opts* o, const osiris_outputs* out, void* stream) {
  if (!cam || !out) return OSIRIS_EINVAL;
  if (int rc = check_opts(o)) return rc;
  const double r_esc = o->r_esc_factor * cam->r0;
  if (disk)
    if (int rc = check_disk(cam->a, o->r_cap_factor, r_esc, r_in, r_out)) return rc;
  if (!is_fin(l0)) return OSIRIS_EINVAL;
  if (int rc = check_spacetime(cam->spacetime, disk)) return rc;
  KernelArgs args;
  std::memset(&args, 0, sizeof(args));
  ReqDev& R = args.single;
  fill_common(R, cam->a, cam->r0, o, o->tol, disk, r_in, r_out, out, l0, cam->spacetime,
              cam->q);
  args.spacetime = cam->spacetime;
  fill_camera(R, cam);
  R.ray_begin = 0;
  args.reqs = nullptr;
  args.n_req = 1;
  args.total_rays = R.n_rays;
  args.stats = reinterpret_cast<unsigned long long*>(o->stats);
  return launch(args, o, stream);
}

}  // namespace

extern "C" {

void osiris_default_opts(osiris_trace_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-10;
  o->max_steps = 1000000;
  o->precision = OSIRIS_FP64;
  o->persistent = 0;
  o->r_cap_factor = 1.01;
  o->r_esc_factor = 1.1;
  o->cell_deg = 10.0;
  o->cell_phase_deg = 0.0;
  o->integrator = OSIRIS_RKCK45;
}

int osiris_init_camera(osiris_camera** out, double a, double r_obs, double incl_deg,
                       double x_min, double x_max, double y_min, double y_max, int32_t nx,
                       int32_t ny) {
  if (!out) return OSIRIS_EINVAL;
  *out = nullptr;
  if (!(a >= 0.0 && a < 1.0)) return OSIRIS_EINVAL;
  if (!is_fin(r_obs) || !(r_obs > 10.0 * horizon(a))) return OSIRIS_EINVAL;
  if (!(incl_deg > 0.0 && incl_deg < 180.0)) return OSIRIS_EINVAL;
  if (!is_fin(x_min) || !is_fin(x_max) || !is_fin(y_min) || !is_fin(y_max)) return OSIRIS_EINVAL;
  if (!(x_min < x_max) || !(y_min < y_max)) return OSIRIS_EINVAL;
  if (nx < 1 || ny < 1) return OSIRIS_EINVAL;
  const double xm = std::fmax(std::fabs(x_min), std::fabs(x_max));
  const double ym = std::fmax(std::fabs(y_min), std::fabs(y_max));
  if (!(xm * xm + ym * ym < r_obs * r_obs)) return OSIRIS_EINVAL;

  osiris_camera* c = new (std::nothrow) osiris_camera;
  if (!c) return OSIRIS_ENOMEM;
  c->spacetime = OSIRIS_SPACETIME_KERR;
  c->q = 0.0;
  c->a = a;
  c->r0 = r_obs;
  c->incl_deg = incl_deg;
  c->th0 = incl_deg * kPi / 180.0;
  c->x_min = x_min;
  c->x_max = x_max;
  c->y_min = y_min;
  c->y_max = y_max;
  c->nx = nx;
  c->ny = ny;
  // Metric at the observer (Eq. Kerr), with the identity
  // g_tphi^2 - g_tt g_phph = Delta sin^2(theta) for A_t of Eq. matrix.
  const double r = r_obs, s = std::sin(c->th0), co = std::cos(c->th0);
  const double s2 = s * s;
  const double Sigma = r * r + a * a * co * co;
  const double Delta = r * r - 2.0 * r + a * a;
  const double rho2 = r * r + a * a;
  const double g_tph = -2.0 * a * r * s2 / Sigma;
  const double g_phph = s2 * (rho2 * rho2 - a * a * Delta * s2) / Sigma;
  const double sq_phph = std::sqrt(g_phph);
  c->inv_At = std::sqrt(Delta * s2 / g_phph);
  c->e_x = g_tph / (r * sq_phph);
  c->l_x = -sq_phph / r;
  c->pth_y = std::sqrt(Sigma) / r;
  c->grr = Sigma / Delta;
  *out = c;
  return OSIRIS_OK;
}

int osiris_init_camera_q(osiris_camera** out, double q, double r_obs, double incl_deg,
                         double x_min, double x_max, double y_min, double y_max, int32_t nx,
                         int32_t ny) {
  if (!out) return OSIRIS_EINVAL;
  *out = nullptr;
  if (!is_fin(q) || !(q > -1.0)) return OSIRIS_EINVAL;
  // validate the image plane with the Kerr a = 0 checks (same r_obs > 20 bound)
  osiris_camera* tmp = nullptr;
  if (int rc = osiris_init_camera(&tmp, 0.0, r_obs, incl_deg, x_min, x_max, y_min, y_max, nx,
                                  ny))
    return rc;
  tmp->spacetime = OSIRIS_SPACETIME_QMETRIC;
  tmp->q = q;
  // observer terms of the initial momenta on the static q-metric (g_tphi = 0,
  // so A_t = 1/sqrt(-g_tt)) at (r_obs, theta0)
  const double r = r_obs, s = std::sin(tmp->th0);
  const double k = q * (2.0 + q);
  const double f = 1.0 - 2.0 / r;
  const double X = 1.0 + s * s / (r * r - 2.0 * r);
  const double g_tt = -std::pow(f, 1.0 + q);
  const double g_rr = std::pow(f, -1.0 - q) * std::pow(X, -k);
  const double g_thth = std::pow(f, -q) * r * r * std::pow(X, -k);
  const double g_phph = std::pow(f, -q) * r * r * s * s;
  tmp->inv_At = std::sqrt(-g_tt);
  tmp->e_x = 0.0;
  tmp->l_x = -std::sqrt(g_phph) / r;
  tmp->pth_y = std::sqrt(g_thth) / r;
  tmp->grr = g_rr;
  *out = tmp;
  return OSIRIS_OK;
}

void osiris_destroy_camera(osiris_camera* cam) { delete cam; }

int64_t osiris_camera_rays(const osiris_camera* cam) {
  return cam ? static_cast<int64_t>(cam->nx) * cam->ny : 0;
}

int osiris_trace(const osiris_camera* cam, const osiris_trace_opts* opts,
                 const osiris_outputs* out, void* cuda_stream) {
  return run_camera(cam, OSIRIS_DISK_NONE, 0.0, 0.0, 0.0, opts, out, cuda_stream);
}

int osiris_render_disk(const osiris_camera* cam, double r_in, double r_out,
                       const osiris_trace_opts* opts, const osiris_outputs* out,
                       void* cuda_stream) {
  return run_camera(cam, OSIRIS_DISK_KEPLERIAN, r_in, r_out, 0.0, opts, out, cuda_stream);
}

int osiris_render_disk_l0(const osiris_camera* cam, double r_in, double r_out, double l0,
                          const osiris_trace_opts* opts, const osiris_outputs* out,
                          void* cuda_stream) {
  return run_camera(cam, OSIRIS_DISK_CONSTANT_L, r_in, r_out, l0, opts, out, cuda_stream);
}

size_t osiris_workspace_bytes(int32_t n_requests) {
  if (n_requests < 1) n_requests = 1;
  return osiris_impl::kQueueBytes + sizeof(ReqDev) * static_cast<size_t>(n_requests);
}

int osiris_trace_batch(const osiris_request* reqs, int32_t n, const osiris_trace_opts* o,
                       void* cuda_stream) {
  if (!reqs || n < 1 || n > 65536) return OSIRIS_EINVAL;
  if (int rc = check_opts(o)) return rc;
  if (!o->workspace || o->workspace_bytes < osiris_workspace_bytes(n)) return OSIRIS_ENOMEM;
  std::vector<ReqDev> table;
  try {
    table.resize(static_cast<size_t>(n));
  } catch (...) {  // no exception crosses the C interface
    return OSIRIS_ENOMEM;
  }
  int64_t begin = 0;
  if (int rc = build_table(reqs, n, o, table.data(), &begin)) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  char* ws = static_cast<char*>(o->workspace);
  ReqDev* dev_table = reinterpret_cast<ReqDev*>(ws + osiris_impl::kQueueBytes);
  if (cudaMemcpyAsync(dev_table, table.data(), sizeof(ReqDev) * table.size(),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return OSIRIS_ECUDA;
  KernelArgs args;
  std::memset(&args, 0, sizeof(args));
  args.reqs = dev_table;
  args.n_req = n;
  args.spacetime = reqs[0].camera->spacetime;
  args.total_rays = begin;
  args.stats = reinterpret_cast<unsigned long long*>(o->stats);
  return launch(args, o, cuda_stream);
}

int osiris_trace_states_ex(int32_t spacetime, double param, double r_obs, double mass2,
                           const double* states, const double* E, const double* L, int64_t n,
                           int32_t disk, double r_in, double r_out, const osiris_trace_opts* o,
                           const osiris_outputs* out, void* cuda_stream) {
  if (!out || n < 0) return OSIRIS_EINVAL;
  if (n > 0 && (!states || !E || !L)) return OSIRIS_EINVAL;
  if (!is_fin(r_obs) || !(r_obs > 0.0) || !is_fin(mass2) || mass2 < 0.0) return OSIRIS_EINVAL;
  double a = 0.0, q = 0.0;
  if (spacetime == OSIRIS_SPACETIME_KERR) {
    if (!(param >= 0.0 && param < 1.0)) return OSIRIS_EINVAL;
    a = param;
  } else if (spacetime == OSIRIS_SPACETIME_QMETRIC) {
    if (!is_fin(param) || !(param > -1.0)) return OSIRIS_EINVAL;
    q = param;
  } else {
    return OSIRIS_EINVAL;
  }
  if (int rc = check_opts(o)) return rc;
  if (int rc = check_spacetime(spacetime, disk)) return rc;
  if (disk)
    if (int rc = check_disk(a, o->r_cap_factor, o->r_esc_factor * r_obs, r_in, r_out)) return rc;
  KernelArgs args;
  std::memset(&args, 0, sizeof(args));
  ReqDev& R = args.single;
  fill_common(R, a, r_obs, o, o->tol, disk ? OSIRIS_DISK_KEPLERIAN : OSIRIS_DISK_NONE, r_in,
              r_out, out, 0.0, spacetime, q, mass2);
  R.explicit_states = 1;
  R.states = states;
  R.E = E;
  R.L = L;
  R.nx = 1;
  R.ny = 1;
  R.n_rays = n;
  R.ray_begin = 0;
  R.pixel_offset = 0;
  args.n_req = 1;
  args.spacetime = spacetime;
  args.total_rays = n;
  args.stats = reinterpret_cast<unsigned long long*>(o->stats);
  return launch(args, o, cuda_stream);
}

int osiris_trace_states(double a, double r_obs, const double* states, const double* E,
                        const double* L, int64_t n, int32_t disk, double r_in, double r_out,
                        const osiris_trace_opts* o, const osiris_outputs* out,
                        void* cuda_stream) {
  return osiris_trace_states_ex(OSIRIS_SPACETIME_KERR, a, r_obs, 0.0, states, E, L, n, disk,
                                r_in, r_out, o, out, cuda_stream);
}

int osiris_copy_outputs_to_host(const osiris_outputs* dev, const osiris_outputs* host, int64_t n,
                                void* cuda_stream) {
  if (!dev || !host || n < 0) return OSIRIS_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  auto cp = [&](void* h, const void* d, size_t elem) -> bool {
    if (!h || !d || n == 0) return true;
    return cudaMemcpyAsync(h, d, elem * static_cast<size_t>(n), cudaMemcpyDeviceToHost, s) ==
           cudaSuccess;
  };
  bool ok = cp(host->status, dev->status, 1) && cp(host->r, dev->r, 8) &&
            cp(host->theta, dev->theta, 8) && cp(host->phi, dev->phi, 8) &&
            cp(host->max_abs_H, dev->max_abs_H, 8) && cp(host->steps, dev->steps, 4) &&
            cp(host->cell_i, dev->cell_i, 2) && cp(host->cell_j, dev->cell_j, 2) &&
            cp(host->parity, dev->parity, 1) && cp(host->g, dev->g, 8) &&
            cp(host->intensity, dev->intensity, 8) && cp(host->r_hit, dev->r_hit, 8);
  return ok ? OSIRIS_OK : OSIRIS_ECUDA;
}

double osiris_isco(double a) {
  // Bardeen, Press & Teukolsky (1972), prograde orbit, M = 1.
  const double z1 =
      1.0 + std::cbrt(1.0 - a * a) * (std::cbrt(1.0 + a) + std::cbrt(1.0 - a));
  const double z2 = std::sqrt(3.0 * a * a + z1 * z1);
  return 3.0 + z2 - std::sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2));
}

double osiris_horizon(double a) { return horizon(a); }

int osiris_pipe_probe(int32_t precision, int32_t op, int64_t n_threads, int32_t iters,
                      double* dev_out, double* flops, void* cuda_stream) {
  if (!dev_out || n_threads < 256 || n_threads % 256 != 0 || iters < 1) return OSIRIS_EINVAL;
  if (n_threads / 256 > 0x7fffffff) return OSIRIS_EINVAL;
  if (precision != OSIRIS_FP64 && precision != OSIRIS_MIXED) return OSIRIS_EINVAL;
  if (op < 0 || op >= osiris_impl::kProbeOps) return OSIRIS_EINVAL;
  if (flops)
    *flops = (op == 0 ? 2.0 : 1.0) * osiris_impl::kProbeFlopsPerThreadIter *
             static_cast<double>(iters) * static_cast<double>(n_threads);
  return cuda_rc(
      osiris_impl::launch_pipe_probe(precision, op, n_threads, iters, dev_out, cuda_stream));
}

int64_t osiris_pipe_probe_threads(int32_t precision, int32_t op) {
  if (precision != OSIRIS_FP64 && precision != OSIRIS_MIXED) return OSIRIS_EINVAL;
  if (op < 0 || op >= osiris_impl::kProbeOps) return OSIRIS_EINVAL;
  int sms = 0, per_sm = 0;
  if (sm_count(&sms) != OSIRIS_OK) return OSIRIS_ECUDA;
  if (osiris_impl::probe_resident_blocks(precision, op, &per_sm) != 0 || per_sm < 1)
    return OSIRIS_ECUDA;
  return static_cast<int64_t>(sms) * per_sm * 256;
}

int osiris_fma_probe(int32_t precision, int64_t n_threads, int32_t iters, double* dev_out,
                     double* flops, void* cuda_stream) {
  return osiris_pipe_probe(precision, 0, n_threads, iters, dev_out, flops, cuda_stream);
}

int osiris_stream_wait(void* cuda_stream, double timeout_s) {
  if (!is_fin(timeout_s) || timeout_s < 0.0) return OSIRIS_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(s);
    if (e == cudaSuccess) return OSIRIS_OK;
    if (e != cudaErrorNotReady) return OSIRIS_ECUDA;
    const std::chrono::duration<double> dt = std::chrono::steady_clock::now() - t0;
    if (dt.count() >= timeout_s) return OSIRIS_ETIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

const char* osiris_strerror(int code) {
  switch (code) {
    case OSIRIS_OK: return "ok";
    case OSIRIS_EINVAL: return "invalid argument";
    case OSIRIS_ECUDA: return "CUDA runtime error";
    case OSIRIS_ENOMEM: return "workspace too small or missing";
    case OSIRIS_ETIMEOUT: return "timed out";
    default: return "unknown error";
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free batched trace (osiris_trace_batch_static): the workspace of
// osiris_trace_batch is replaced by one fixed array in device memory.
// ---------------------------------------------------------------------------
namespace {

constexpr int kStaticMaxDevices = 64;
constexpr size_t kStaticBytes =
    osiris_impl::kQueueBytes + sizeof(ReqDev) * static_cast<size_t>(OSIRIS_STATIC_MAX_REQUESTS);

// Queue counter (first 256 bytes) and request table; one copy per device.
__device__ __align__(256) unsigned char g_static_workspace[kStaticBytes];

std::mutex g_static_mutex;                      // guards the two arrays below
void* g_static_address[kStaticMaxDevices] = {};  // device address, per device
ReqDev g_static_table[OSIRIS_STATIC_MAX_REQUESTS];  // host staging of the table

// Device address of g_static_workspace on the current device, looked up once
// per device. Host code must not use the symbol itself as an address.
int static_workspace_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OSIRIS_ECUDA;
  if (dev < 0 || dev >= kStaticMaxDevices) return OSIRIS_EINVAL;
  if (g_static_address[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_workspace) != cudaSuccess || p == nullptr)
      return OSIRIS_ECUDA;
    g_static_address[dev] = p;
  }
  *out = g_static_address[dev];
  return OSIRIS_OK;
}

}  // namespace

extern "C" int osiris_trace_batch_static(const osiris_request* reqs, int32_t n,
                                         const osiris_trace_opts* opts, void* cuda_stream) {
  if (!reqs || !opts || n < 1 || n > OSIRIS_STATIC_MAX_REQUESTS) return OSIRIS_EINVAL;
  osiris_trace_opts o = *opts;
  o.workspace = nullptr;
  o.workspace_bytes = 0;
  if (int rc = check_opts(&o)) return rc;

  std::lock_guard<std::mutex> lock(g_static_mutex);
  int64_t begin = 0;
  if (int rc = build_table(reqs, n, &o, g_static_table, &begin)) return rc;
  void* base = nullptr;
  if (int rc = static_workspace_address(&base)) return rc;
  char* ws = static_cast<char*>(base);
  ReqDev* dev_table = reinterpret_cast<ReqDev*>(ws + osiris_impl::kQueueBytes);
  // Pageable source: the call returns once the table has been staged, so the
  // host table may be refilled by the next call.
  if (cudaMemcpyAsync(dev_table, g_static_table, sizeof(ReqDev) * static_cast<size_t>(n),
                      cudaMemcpyHostToDevice, static_cast<cudaStream_t>(cuda_stream)) !=
      cudaSuccess)
    return OSIRIS_ECUDA;
  KernelArgs args;
  std::memset(&args, 0, sizeof(args));
  args.reqs = dev_table;
  args.n_req = n;
  args.spacetime = reqs[0].camera->spacetime;
  args.total_rays = begin;
  args.stats = reinterpret_cast<unsigned long long*>(o.stats);
  o.workspace = base;  // launch() clears the queue counter at its head
  o.workspace_bytes = kStaticBytes;
  return launch(args, &o, cuda_stream);
}

// ---------------------------------------------------------------------------
// Batch plans: the three operations of a batched persistent launch (request
// table upload, queue reset, trace kernel) recorded once as a CUDA graph and
// replayed per batch. The upload always copies the plan's whole staging table
// (max_requests entries of a few hundred bytes), so only the kernel arguments
// and the grid change between batches; they are patched into the
// instantiated graph.
// ---------------------------------------------------------------------------
struct osiris_batch_plan {
  osiris_trace_opts opts;  // fixed per plan (workspace, stats, launch shape, defaults)
  int32_t max_requests = 0;
  int32_t spacetime = OSIRIS_SPACETIME_KERR;
  int block = 0;
  int64_t full_grid = 0;
  ReqDev* staging = nullptr;    // pinned host copy of the request table
  ReqDev* dev_table = nullptr;  // inside opts.workspace
  cudaEvent_t copied = nullptr;  // recorded by the graph once the table is uploaded
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t kernel_node = nullptr;
  cudaKernelNodeParams kernel{};  // function, block and shared memory of the launch
};

namespace {

void release(osiris_batch_plan* p) {
  if (!p) return;
  if (p->copied) cudaEventSynchronize(p->copied);  // the last upload reads staging
  if (p->exec) cudaGraphExecDestroy(p->exec);    // in-flight launches still complete
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->copied) cudaEventDestroy(p->copied);
  if (p->staging) cudaFreeHost(p->staging);
  delete p;
}

// Record upload -> event -> queue reset -> kernel on a private stream.
int record_plan(osiris_batch_plan* p) {
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return OSIRIS_ECUDA;
  int rc = OSIRIS_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaStreamDestroy(cs);
    return OSIRIS_ECUDA;
  }
  KernelArgs args;
  std::memset(&args, 0, sizeof(args));
  args.reqs = p->dev_table;
  args.n_req = 1;
  args.spacetime = p->spacetime;
  args.total_rays = 1;
  args.stats = reinterpret_cast<unsigned long long*>(p->opts.stats);
  args.queue = static_cast<unsigned long long*>(p->opts.workspace);
  set_granularity(args, &p->opts);
  // An external event record node: the host waits on it before rewriting the
  // staging table.
  if (cudaMemcpyAsync(p->dev_table, p->staging,
                      sizeof(ReqDev) * static_cast<size_t>(p->max_requests),
                      cudaMemcpyHostToDevice, cs) != cudaSuccess ||
      cudaEventRecordWithFlags(p->copied, cs, cudaEventRecordExternal) != cudaSuccess ||
      cudaMemsetAsync(args.queue, 0, sizeof(unsigned long long), cs) != cudaSuccess ||
      launcher_of(&p->opts)(args, Kernel::kPersistent, p->opts.integrator, 1, p->block, cs) != 0)
    rc = OSIRIS_ECUDA;
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(cs, &g) != cudaSuccess) rc = OSIRIS_ECUDA;
  cudaStreamDestroy(cs);
  p->graph = g;
  if (rc != OSIRIS_OK) return rc;

  size_t count = 0;
  if (cudaGraphGetNodes(g, nullptr, &count) != cudaSuccess) return OSIRIS_ECUDA;
  std::vector<cudaGraphNode_t> nodes;
  try {
    nodes.resize(count);
  } catch (...) {
    return OSIRIS_ENOMEM;
  }
  if (count == 0 || cudaGraphGetNodes(g, nodes.data(), &count) != cudaSuccess)
    return OSIRIS_ECUDA;
  for (cudaGraphNode_t n : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(n, &t) != cudaSuccess) return OSIRIS_ECUDA;
    if (t == cudaGraphNodeTypeKernel) {
      p->kernel_node = n;
      if (cudaGraphKernelNodeGetParams(n, &p->kernel) != cudaSuccess) return OSIRIS_ECUDA;
    }
  }
  if (!p->kernel_node) return OSIRIS_ECUDA;
  if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) return OSIRIS_ECUDA;
  return OSIRIS_OK;
}

}  // namespace

extern "C" {

int osiris_batch_plan_create(osiris_batch_plan** out, int32_t max_requests, int32_t spacetime,
                             const osiris_trace_opts* opts) {
  if (!out || !opts || max_requests < 1 || max_requests > 65536) return OSIRIS_EINVAL;
  *out = nullptr;
  if (int rc = check_opts(opts)) return rc;
  if (int rc = check_spacetime(spacetime, OSIRIS_DISK_NONE)) return rc;
  if (!opts->workspace || opts->workspace_bytes < osiris_workspace_bytes(max_requests))
    return OSIRIS_ENOMEM;
  osiris_batch_plan* p = new (std::nothrow) osiris_batch_plan;
  if (!p) return OSIRIS_ENOMEM;
  p->opts = *opts;
  p->opts.persistent = 1;
  p->max_requests = max_requests;
  p->spacetime = spacetime;
  p->dev_table = reinterpret_cast<ReqDev*>(static_cast<char*>(opts->workspace) +
                                           osiris_impl::kQueueBytes);
  int rc = persistent_shape(&p->opts, spacetime, &p->block, &p->full_grid);
  if (rc == OSIRIS_OK &&
      cudaMallocHost(&p->staging, sizeof(ReqDev) * static_cast<size_t>(max_requests)) !=
          cudaSuccess) {
    p->staging = nullptr;
    rc = OSIRIS_ENOMEM;
  }
  if (rc == OSIRIS_OK &&
      cudaEventCreateWithFlags(&p->copied, cudaEventDisableTiming) != cudaSuccess) {
    p->copied = nullptr;
    rc = OSIRIS_ECUDA;
  }
  if (rc == OSIRIS_OK) {
    std::memset(p->staging, 0, sizeof(ReqDev) * static_cast<size_t>(max_requests));
    rc = record_plan(p);
  }
  if (rc != OSIRIS_OK) {
    release(p);
    return rc;
  }
  *out = p;
  return OSIRIS_OK;
}

int osiris_batch_plan_launch(osiris_batch_plan* p, const osiris_request* reqs, int32_t n,
                             void* cuda_stream) {
  if (!p || !reqs || n < 1 || n > p->max_requests) return OSIRIS_EINVAL;
  if (!reqs[0].camera || reqs[0].camera->spacetime != p->spacetime) return OSIRIS_EINVAL;
  // The previous batch's upload must have read the staging table.
  if (cudaEventSynchronize(p->copied) != cudaSuccess) return OSIRIS_ECUDA;
  int64_t total = 0;
  if (int rc = build_table(reqs, n, &p->opts, p->staging, &total)) return rc;
  if (total == 0) return OSIRIS_OK;
  KernelArgs args;
  std::memset(&args, 0, sizeof(args));
  args.reqs = p->dev_table;
  args.n_req = n;
  args.spacetime = p->spacetime;
  args.total_rays = total;
  args.stats = reinterpret_cast<unsigned long long*>(p->opts.stats);
  args.queue = static_cast<unsigned long long*>(p->opts.workspace);
  set_granularity(args, &p->opts);
  const int64_t per_block = static_cast<int64_t>(p->block) * args.rays_per_lane;
  int64_t grid = (total + per_block - 1) / per_block;
  if (grid > p->full_grid) grid = p->full_grid;
  cudaKernelNodeParams k = p->kernel;
  void* argv[] = {&args};
  k.gridDim = dim3(static_cast<unsigned>(grid), 1, 1);
  k.kernelParams = argv;
  k.extra = nullptr;
  if (cudaGraphExecKernelNodeSetParams(p->exec, p->kernel_node, &k) != cudaSuccess ||
      cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess)
    return OSIRIS_ECUDA;
  return OSIRIS_OK;
}

void osiris_batch_plan_destroy(osiris_batch_plan* p) { release(p); }

}  // extern "C"
