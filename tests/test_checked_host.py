"""The index checks of the bounds-checked build (csrc/checked.cuh), compiled
as host C++: every planted bad index (a ray past the launch's queue, a request
index outside the table, a ray outside its request's range, a pixel or state
index outside the outputs) gives its code, and every valid index of a small
ragged batch passes. The GPU test (test_gpu_checked.py) runs the whole
checked library and finds no failure on valid launches."""
import subprocess

from _df_host import build

HARNESS = r"""
#include "checked.cuh"
using namespace osiris_impl;
int main() {
  long long v[4];
  while (std::fscanf(stdin, "%lld %lld %lld %lld", v, v + 1, v + 2, v + 3) == 4) {
    // g total req n_req | ray_begin n_rays local limit (second stage if first passes)
    unsigned c = check_ray_request(v[0], v[1], (int)v[2], (int)v[3]);
    long long w[4];
    if (std::fscanf(stdin, "%lld %lld %lld %lld", w, w + 1, w + 2, w + 3) != 4) return 1;
    if (c == CHECK_OK) c = check_ray_pixel(v[0], w[0], w[1], w[2], w[3]);
    std::printf("%u %llu\n", c, check_word(c, v[0]));
  }
  return 0;
}
"""


def _run(exe, rows):
    text = "\n".join(" ".join(str(x) for x in r) for r in rows) + "\n"
    out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True)
    return [tuple(int(x) for x in ln.split()) for ln in out.stdout.split("\n") if ln]


def test_planted_bad_indices_are_caught(tmp_path_factory):
    exe = build(tmp_path_factory, "checked", HARNESS, device_shims=True)
    # (g, total, req, n_req, ray_begin, n_rays, local, limit) -> code
    cases = [
        ((5, 10, 0, 1, 0, 10, 5, 10), 0),
        ((10, 10, 0, 1, 0, 10, 10, 10), 1),       # one past the queue
        ((-1, 10, 0, 1, 0, 10, -1, 10), 1),       # negative ray
        ((3, 10, 2, 2, 0, 10, 3, 10), 2),         # request index = table size
        ((3, 10, -1, 2, 0, 10, 3, 10), 2),        # negative request index
        ((3, 10, 1, 2, 4, 6, 0, 6), 3),           # ray before its request's range
        ((9, 10, 0, 2, 0, 9, 9, 9), 3),           # ray after its request's range
        ((7, 10, 1, 2, 4, 6, 6, 6), 4),           # pixel index = nx ny (bad offset)
        ((7, 10, 1, 2, 4, 6, -2, 6), 4),          # negative pixel index
    ]
    got = _run(exe, [args for args, _ in cases])
    for (args, code), (c, word) in zip(cases, got):
        assert c == code, (args, c)
        if code:
            assert word >> 56 == code and (word & ((1 << 56) - 1)) == (args[0] & ((1 << 56) - 1))
        else:
            assert word == args[0]


def test_every_index_of_a_ragged_batch_passes(tmp_path_factory):
    exe = build(tmp_path_factory, "checked_ok", HARNESS, device_shims=True)
    # three requests: a 2x3 render, a pixel range [5, 12) of a 5x3 render, a 1x1 render
    reqs = [(0, 6, 0, 6), (6, 7, 5, 15), (13, 1, 0, 1)]  # ray_begin, n_rays, offset, nx*ny
    total = 14
    rows = []
    for k, (begin, n, off, limit) in enumerate(reqs):
        for g in range(begin, begin + n):
            rows.append((g, total, k, len(reqs), begin, n, g - begin + off, limit))
    assert all(c == 0 for c, _ in _run(exe, rows))
