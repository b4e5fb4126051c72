// Bounds checks of the OSIRIS_CHECKED build (the stand-in for a memory
// checker). Before a lane reads anything of a ray, the checked kernels test
// the ray's queue index, its request index, and its pixel (or explicit-state)
// index against the sizes the host validated; a failed check skips the ray
// (the lane stays idle) and is counted in the caller's stats array instead of
// trapping:
//   stats[OSIRIS_STAT_CHECK_FAILS]  number of failed checks
//   stats[OSIRIS_STAT_CHECK_WORST]  max over failures of (code << 56) | ray
// The index tests are plain integer functions, so they also compile as host
// C++ (the CPU tests plant bad indices there).
#pragma once

#include <cstdint>

#include "osiris.h"

namespace osiris_impl {

enum : unsigned {
  CHECK_OK = 0,
  CHECK_QUEUE = 1,    // ray index outside [0, total rays of the launch)
  CHECK_REQUEST = 2,  // request index outside [0, requests of the launch)
  CHECK_RANGE = 3,    // ray not inside its request's range of the queue
  CHECK_PIXEL = 4,    // pixel / state index outside the request's outputs
};

// First stage: indices that are valid before the request table is read.
__host__ __device__ inline unsigned check_ray_request(int64_t g, int64_t total, int req,
                                                      int n_req) {
  if (g < 0 || g >= total) return CHECK_QUEUE;
  if (req < 0 || req >= n_req) return CHECK_REQUEST;
  return CHECK_OK;
}

// Second stage, with the request's entries: g in [ray_begin, ray_begin +
// n_rays) and the output index local in [0, limit) (limit = nx ny for a
// pixel render, the number of explicit states otherwise).
__host__ __device__ inline unsigned check_ray_pixel(int64_t g, int64_t ray_begin, int64_t n_rays,
                                                    int64_t local, int64_t limit) {
  if (g < ray_begin || g - ray_begin >= n_rays) return CHECK_RANGE;
  if (local < 0 || local >= limit) return CHECK_PIXEL;
  return CHECK_OK;
}

__host__ __device__ inline unsigned long long check_word(unsigned code, int64_t g) {
  return ((unsigned long long)code << 56) | ((unsigned long long)g & ((1ull << 56) - 1));
}

}  // namespace osiris_impl
