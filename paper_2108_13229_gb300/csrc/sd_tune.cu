// sd_tune.cu -- autotuner for the launch shape and the multigrid hierarchy.
//
// Which smoothing tile, how deep a V-cycle and how many Chebyshev steps give
// the shortest time step depends on the grid size (how many CTAs fill the
// 152 SMs, how many levels sit below the fused coarse cycle) and on the
// device, and the iteration count moves with the smoother as well, so the
// choice is measured rather than modelled: every candidate in a small grid of
// (tile_rows, coarsest, cheb_degree) runs the same time steps from the same
// initial state, and the one with the smallest device time per step whose
// steps all converged wins.  Results are kept in a plain-text cache file, one
// line per (device, grid size, solver mode), so a size is tuned once per
// machine.  Host code only, built on the public C ABI.
#include "../../include/sd.h"

#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace {

std::mutex g_cache_mu;

struct Key {
  std::string dev;
  int n, precision, precond, darcy_coupled, restart, bc, coupling;
  double rtol;
};

std::string device_tag() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string s = p.name;
  for (char& c : s)
    if (c == ' ' || c == '\t') c = '_';
  char buf[64];
  std::snprintf(buf, sizeof(buf), "_sm%d.%d_x%d", p.major, p.minor, p.multiProcessorCount);
  return s + buf;
}

// One cache line: "sdtune2 dev n precision precond darcy_coupled restart bc
// coupling rtol tile_rows coarsest cheb_degree ms_per_step".
bool cache_lookup(const char* path, const Key& k, sd_options* o, double* ms) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[512], dev[256];
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    int n, pr, pc, dc, rs, bc, cp, tr, co, cd;
    double rt, t;
    if (std::sscanf(line, "sdtune2 %255s %d %d %d %d %d %d %d %lg %d %d %d %lg", dev, &n, &pr, &pc, &dc, &rs, &bc,
                    &cp, &rt, &tr, &co, &cd, &t) != 13)
      continue;
    if (k.dev != dev || n != k.n || pr != k.precision || pc != k.precond || dc != k.darcy_coupled ||
        rs != k.restart || bc != k.bc || cp != k.coupling || rt != k.rtol)
      continue;
    // a line whose options sd_create would reject (an edited or damaged
    // file) is skipped
    sd_options c = *o;
    c.tile_rows = tr;
    c.coarsest = co;
    c.cheb_degree = cd;
    const sd_grid g{k.n, k.n};
    if (sd_memory_estimate(&g, &c) < 0) continue;
    *o = c;  // the last valid matching line wins
    *ms = t;
    found = true;
  }
  std::fclose(f);
  return found;
}

void cache_store(const char* path, const Key& k, const sd_options& o, double ms) {
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "sdtune2 %s %d %d %d %d %d %d %d %.17g %d %d %d %.6f\n", k.dev.c_str(), k.n, k.precision,
               k.precond, k.darcy_coupled, k.restart, k.bc, k.coupling, k.rtol, o.tile_rows, o.coarsest,
               o.cheb_degree, ms);
  std::fclose(f);
}

// Untimed steps before a candidate is timed: the first steps from the
// initial state take two to three times the iterations of the later ones,
// which would weight the choice towards the start-up transient.
const int kWarm = 4;

// Device time per step of `nsteps` steps after `warm` untimed ones, from a
// fresh instance; negative when setup failed or a step did not converge.
double time_candidate(const sd_grid* grid, double mu, const double* K, double alpha, double dt,
                      const sd_options& o, int warm, int nsteps) {
  sd_handle* h = nullptr;
  if (sd_create(grid, mu, K, alpha, dt, &o, &h) != SD_OK) {
    if (h) sd_destroy(h);
    return -1.0;
  }
  std::vector<sd_step_info> info((size_t)(warm + nsteps));
  const int rc = sd_step(h, warm + nsteps, info.data());
  sd_destroy(h);
  if (rc != SD_OK) return -1.0;
  double ms = 0.0;
  for (int k = warm; k < warm + nsteps; ++k) ms += info[(size_t)k].ms;
  return ms / nsteps;
}

}  // namespace

extern "C" int sd_autotune(const sd_grid* grid, double mu, const double* K, double alpha_bj, double dt,
                           const sd_options* base, int32_t nsteps, const char* cache_path, sd_options* best,
                           double* best_ms) {
  if (!grid || !K || !best || nsteps < 1 || grid->nx != grid->ny || grid->nx < 2) return SD_E_INVAL;
  sd_options b;
  sd_options_default(&b);
  if (base) b = *base;
  Key key{device_tag(), grid->nx, b.precision, b.precond, b.darcy_coupled, b.restart, b.bc, b.coupling, b.rtol};
  if (cache_path && cache_path[0]) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    sd_options o = b;
    double ms = 0.0;
    if (cache_lookup(cache_path, key, &o, &ms)) {
      *best = o;
      if (best_ms) *best_ms = ms;
      return SD_OK;
    }
  }
  // the candidate grid: tile height only matters for the FP32 tiled smoother
  const bool tiles = b.precision == SD_MIXED && b.tile;
  const int rows[3] = {0, 16, 8};  // 0: by level size (4, 8 or 16 rows)
  const int coarse[3] = {4, 8, 16};
  const int degree[3] = {3, 2, 4};
  double best_t = -1.0;
  sd_options win = b;
  for (int r = 0; r < (tiles ? 3 : 1); ++r)
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) {
        sd_options o = b;
        o.tile_rows = tiles ? rows[r] : b.tile_rows;
        o.coarsest = coarse[c];
        o.cheb_degree = degree[d];
        if (c > 0 && coarse[c - 1] >= grid->nx) continue;  // already a one-level hierarchy
        const double t = time_candidate(grid, mu, K, alpha_bj, dt, o, kWarm, nsteps);
        if (t > 0 && (best_t < 0 || t < best_t)) {
          best_t = t;
          win = o;
        }
      }
  if (best_t < 0) return SD_E_NOCONV;
  *best = win;
  if (best_ms) *best_ms = best_t;
  if (cache_path && cache_path[0]) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    cache_store(cache_path, key, win, best_t);
  }
  return SD_OK;
}
