// Autotuner for batched solves (no counterpart in the paper): times the
// launch configurations of bo_solve_batched on the caller's own batch
// (per-kernel stream launches, per-column CUDA graphs per realisation, or
// one graph per column for the whole batch in lockstep, and the width of
// the stream pool) and keeps the winner in a small JSON cache keyed by the
// batch's shape, so that later runs apply it without timing.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "bo_internal.cuh"

namespace {

// batch shape -> key: counts and size classes (log2 buckets), precision, restart
std::string tune_key(bo_prec* const* P, int nreal, const bo_solve_opts* o) {
  int64_t total = 0, largest = 0;
  int fp32 = 0;
  for (int r = 0; r < nreal; ++r) {
    const int64_t n = P[r]->mat->g.N;
    total += n;
    largest = std::max(largest, n);
    fp32 += P[r]->fp32 ? 1 : 0;
  }
  auto lg = [](int64_t v) { return v > 0 ? (int)std::floor(std::log2((double)v)) : 0; };
  std::ostringstream k;
  k << "batch" << nreal << "_cells2^" << lg(total) << "_max2^" << lg(largest) << "_fp32x" << fp32 << "_m"
    << o->restart;
  return k.str();
}

// the cache: one line per entry, "key": [launch_mode, streams, ms, amg_cells,
// amg_threads] (entries of three values, from before the tile search, keep
// the default tile)
std::map<std::string, std::vector<double>> read_cache(const char* path) {
  std::map<std::string, std::vector<double>> out;
  if (!path) return out;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t a = line.find('"'), b = line.find('"', a + 1), l = line.find('['), r = line.find(']');
    if (a == std::string::npos || b == std::string::npos || l == std::string::npos || r == std::string::npos) continue;
    std::vector<double> v;
    std::stringstream ss(line.substr(l + 1, r - l - 1));
    std::string tok;
    while (std::getline(ss, tok, ',')) v.push_back(std::atof(tok.c_str()));
    if (v.size() == 3) v.insert(v.end(), {1.0, 256.0});
    if (v.size() == 5) out[line.substr(a + 1, b - a - 1)] = v;
  }
  return out;
}

bool write_cache(const char* path, const std::map<std::string, std::vector<double>>& c) {
  if (!path) return true;
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream f(tmp);
    if (!f) return false;
    f << "{\n";
    size_t i = 0;
    for (const auto& kv : c) {
      f << "  \"" << kv.first << "\": [" << (int)kv.second[0] << ", " << (int)kv.second[1] << ", " << kv.second[2]
        << ", " << (int)kv.second[3] << ", " << (int)kv.second[4] << "]" << (++i < c.size() ? "," : "") << "\n";
    }
    f << "}\n";
  }
  return std::rename(tmp.c_str(), path) == 0;
}

void apply(bo_prec* const* P, int nreal, int mode, int streams, int cells = 1, int threads = 256) {
  for (int r = 0; r < nreal; ++r) {
    P[r]->launch_mode = mode;
    bo_prec_set_amg_tile(P[r], cells, threads);
  }
  bo::g_pool_width.store(std::max(1, std::min(bo::kMaxPoolStreams, streams)));
}

}  // namespace

extern "C" {

int bo_autotune_batched(bo_prec* const* P, int nreal, const double* const* b, double* const* x,
                        const bo_solve_opts* opts, const char* cache_path, bo_tune_result* out) {
  if (!P || !b || !x || !opts || nreal < 1) return BO_ERR_ARG;
  const std::string key = tune_key(P, nreal, opts);
  auto cache = read_cache(cache_path);
  auto it = cache.find(key);
  if (it != cache.end()) {
    const std::vector<double>& v = it->second;
    apply(P, nreal, (int)v[0], (int)v[1], (int)v[3], (int)v[4]);
    if (out) {
      std::memset(out, 0, sizeof(*out));
      out->launch_mode = (int)v[0];
      out->streams = (int)v[1];
      out->best_ms = v[2];
      out->from_cache = 1;
      out->amg_cells = (int)v[3];
      out->amg_threads = (int)v[4];
    }
    return BO_OK;
  }
  const int modes[3] = {BO_LAUNCH_STREAM, BO_LAUNCH_GRAPH, BO_LAUNCH_BATCH_GRAPH};
  const int widths[3] = {4, 8, 16};
  bo_solve_opts o = *opts;
  o.x0_is_zero = 1;
  o.profile = 0;
  double best = 1e300;
  int best_mode = BO_LAUNCH_STREAM, best_w = bo::kMaxPoolStreams;
  double ms[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  int k = 0;
  for (int mi = 0; mi < 3; ++mi)
    for (int wi = 0; wi < 3; ++wi, ++k) {
      apply(P, nreal, modes[mi], widths[wi]);
      // one untimed pass (graph capture, first-touch), then the timed one
      for (int pass = 0; pass < 2; ++pass) {
        const auto t0 = std::chrono::steady_clock::now();
        const int rc = bo_solve_batched(P, nreal, b, x, &o, nullptr);
        const double t = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (rc != BO_OK && rc != BO_ERR_NOT_CONVERGED) return rc;
        if (pass == 1) ms[k] = t;
      }
      if (ms[k] < best) {
        best = ms[k];
        best_mode = modes[mi];
        best_w = widths[wi];
      }
    }
  // the tile of the per-kernel AMG form, which the graph forms run: level-0
  // cells per thread and threads per block, tried with the best form and
  // width (the default, 1 cell and 256 threads, was timed above)
  const int tiles[5][2] = {{2, 256}, {4, 256}, {1, 128}, {2, 128}, {1, 512}};
  double tms[5] = {0, 0, 0, 0, 0};
  int best_cells = 1, best_threads = 256;
  if (best_mode != BO_LAUNCH_STREAM) {
    for (int ti = 0; ti < 5; ++ti) {
      apply(P, nreal, best_mode, best_w, tiles[ti][0], tiles[ti][1]);
      for (int pass = 0; pass < 2; ++pass) {
        const auto t0 = std::chrono::steady_clock::now();
        const int rc = bo_solve_batched(P, nreal, b, x, &o, nullptr);
        const double t = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (rc != BO_OK && rc != BO_ERR_NOT_CONVERGED) return rc;
        if (pass == 1) tms[ti] = t;
      }
      if (tms[ti] < best) {
        best = tms[ti];
        best_cells = tiles[ti][0];
        best_threads = tiles[ti][1];
      }
    }
  }
  apply(P, nreal, best_mode, best_w, best_cells, best_threads);
  cache[key] = {(double)best_mode, (double)best_w, best, (double)best_cells, (double)best_threads};
  const bool wrote = write_cache(cache_path, cache);
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->launch_mode = best_mode;
    out->streams = best_w;
    out->best_ms = best;
    out->from_cache = 0;
    for (int i = 0; i < 9; ++i) out->trial_ms[i] = ms[i];
    out->amg_cells = best_cells;
    out->amg_threads = best_threads;
    for (int i = 0; i < 5; ++i) out->tile_ms[i] = tms[i];
  }
  return wrote ? BO_OK : BO_ERR_ARG;
}

int bo_set_batch_streams(int n) {
  if (n < 1 || n > bo::kMaxPoolStreams) return BO_ERR_ARG;
  bo::g_pool_width.store(n);
  return BO_OK;
}

}  // extern "C"
