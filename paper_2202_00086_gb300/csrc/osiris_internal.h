// Internal layout shared by the host API (osiris_api.cu) and the trace
// kernels (trace_*.cu). Not part of the public interface.
#pragma once

#include <cstddef>
#include <cstdint>

#include "osiris.h"

namespace osiris_impl {

// One render (or one explicit-state batch) as the kernels see it. Lives in
// kernel parameter space for single renders and in the workspace for
// batches. Every quantity the kernels need per ray is precomputed on the host.
struct alignas(16) ReqDev {
  // space-time (M = 1): Kerr with spin a, or the q-metric with quadrupole q
  int32_t spacetime;  // OSIRIS_SPACETIME_*
  double a;
  double q;
  // mass shell: H = H0 (0 for light, -1/2 for massive particles)
  double H0;
  // observer and image plane (Sec. 2.3)
  double r0, th0;
  double x_min, x_span, y_min, y_span;  // centre of pixel i: x_min + (i + 1/2) x_span / nx
  int32_t nx, ny;
  // observer terms of the initial momenta:
  //   E = inv_At + x e_x,  L = x l_x,  p_theta = y pth_y,
  //   p_r = -sqrt(grr (1 - (x^2 + y^2) / r0^2))
  double inv_At, e_x, l_x, pth_y, grr;
  // stopping surfaces (Sec. 4.1, Sec. 5)
  double r_cap, r_esc, r_in, r_out;
  int32_t disk;             // OSIRIS_DISK_* (0: no disk)
  double l0;                // constant-l0 disk
  int32_t explicit_states;  // 1: rays start from states / E / L (test hook)
  const double* states;     // n x 6 rows (t, r, theta, phi, p_r, p_theta)
  const double* E;
  const double* L;
  // integrator
  double tol, h0;
  int64_t max_steps;
  // celestial checkerboard
  double cell_rad, phase_rad, inv_cell;  // inv_cell = 1 / cell_rad
  int32_t n_th_cells, n_ph_cells;
  // position in the launch's global ray queue; pixel index of its first ray
  int64_t ray_begin, n_rays, pixel_offset;
  osiris_outputs out;
};

// Kernel arguments (passed as a __grid_constant__ parameter).
struct KernelArgs {
  const ReqDev* reqs;              // device table (batch); nullptr -> use `single`
  int32_t n_req;
  int32_t spacetime;               // of every request in the launch
  int64_t total_rays;
  unsigned long long* queue;       // persistent grids: next ray index (device)
  unsigned long long* stats;       // optional OSIRIS_STATS_LEN counters (device)
  int32_t rays_per_lane;           // rays a lane claims at once (plain: per thread), >= 1
  int32_t refill_lanes;            // persistent: idle lanes a warp waits for before it
                                   // refills (unless none of its lanes is busy), 1..32
  ReqDev single;
};

constexpr size_t kQueueBytes = 256;  // workspace head: the ray counter

enum class Kernel { kPlain, kPersistent };

// Launchers implemented in the kernel translation units. They return a
// cudaError_t value as int (0 = success).
int launch_trace_fp64(const KernelArgs& args, Kernel kind, int integrator, int grid, int block,
                      void* stream);
int launch_trace_mixed(const KernelArgs& args, Kernel kind, int integrator, int grid, int block,
                       void* stream);
int launch_trace_df64(const KernelArgs& args, Kernel kind, int integrator, int grid, int block,
                      void* stream);
int occupancy_fp64(Kernel kind, int integrator, int spacetime, int block, int* blocks_per_sm);
int occupancy_mixed(Kernel kind, int integrator, int spacetime, int block, int* blocks_per_sm);
int occupancy_df64(Kernel kind, int integrator, int spacetime, int block, int* blocks_per_sm);
// Pipe probes (roofline denominators): 16 chains per thread of one
// operation (0 FMA, 1 multiply, 2 add, 3 multiply as FMA, 4 add as FMA),
// 256 threads per block.
constexpr int kProbeOps = 5;
constexpr int kProbeFlopsPerThreadIter = 16 * 4;  // operations per thread per loop trip
int launch_pipe_probe(int precision, int op, int64_t n_threads, int iters, double* out,
                      void* stream);
int probe_resident_blocks(int precision, int op, int* blocks_per_sm);

}  // namespace osiris_impl
