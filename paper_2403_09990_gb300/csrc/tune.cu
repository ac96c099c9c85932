// Autotuner: launch shapes chosen by measurement and cached per (operation, PURSE kind,
// keypoint-count bucket, sample-count bucket, variant, GPU name).
//
// Operations and their shapes (none changes a result: every walk is one warp's work, the farthest
// sample of a ball is the lowest-index maximum whatever the grid, every pose's distance is its own):
//   walk  -- warps per walk block {8, 4, 2} (purse_sample; variant = sampler + 2 precision);
//   megb  -- samples per thread of the persistent ball kernel, i.e. the blocks per ball
//            (megb_solve; variant = precision);
//   dist  -- resident CTAs per SM of the tensor-core distance kernel (purse_dist modes 1 and 2;
//            variant = passes).
// The cache lives in the process; PURSE_TUNE_CACHE names a file it is loaded from at first use and
// appended to by every tuning call.  A tuning call forces each candidate in turn (thread-local
// override read by the launchers), times it with CUDA events on the caller's stream and stores the
// fastest.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "internal.h"

namespace purse {

namespace {
std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune;
bool g_tune_loaded = false;
thread_local int g_force_op = -1, g_force_cfg = 0;
char g_gpu_name[256] = "";

int bucket_n(int n) {  // ceil(log2 n)
  int b = 0;
  while ((1 << b) < n) ++b;
  return b;
}
int bucket_s(long long s) {  // floor(log2 s)
  int b = 0;
  while (s > 1) s >>= 1, ++b;
  return b;
}

std::string make_key(int op, int kind, int n, long long samples, int variant, const char* gpu) {
  char buf[512];
  std::snprintf(buf, sizeof buf, "%d %d %d %d %d %s", op, kind, bucket_n(n), bucket_s(samples), variant, gpu);
  for (char* c = buf; *c; ++c)
    if (*c == '\n' || *c == '\t') *c = ' ';
  return buf;
}

void load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("PURSE_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[1024];
  while (std::fgets(line, sizeof line, f)) {
    // key fields (5 integers and the GPU name) | cfg ms default_ms
    char* bar = std::strrchr(line, '|');
    if (!bar) continue;
    *bar = 0;
    TuneEntry e{};
    if (std::sscanf(bar + 1, "%d %f %f", &e.cfg, &e.ms, &e.default_ms) != 3) continue;
    std::string key(line);
    while (!key.empty() && key.back() == ' ') key.pop_back();
    g_tune[key] = e;
  }
  std::fclose(f);
}

const char* gpu_name() {
  if (!g_gpu_name[0]) {
    int dev = 0;
    cudaDeviceProp p;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&p, dev) == cudaSuccess)
      std::snprintf(g_gpu_name, sizeof g_gpu_name, "%s", p.name);
    else
      std::snprintf(g_gpu_name, sizeof g_gpu_name, "unknown");
  }
  return g_gpu_name;
}
}  // namespace

bool tune_lookup(int op, int kind, int n, long long samples, int variant, const char* gpu, TuneEntry* out) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  load_locked();
  auto it = g_tune.find(make_key(op, kind, n, samples, variant, gpu));
  if (it == g_tune.end()) return false;
  *out = it->second;
  return true;
}

void tune_store(int op, int kind, int n, long long samples, int variant, const char* gpu, const TuneEntry& e) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  load_locked();
  const std::string key = make_key(op, kind, n, samples, variant, gpu);
  g_tune[key] = e;
  const char* path = std::getenv("PURSE_TUNE_CACHE");
  if (path && *path) {
    if (FILE* f = std::fopen(path, "a")) {
      std::fprintf(f, "%s | %d %.6g %.6g\n", key.c_str(), e.cfg, e.ms, e.default_ms);
      std::fclose(f);
    }
  }
}

int tuned_config(int op, int kind, int n, long long samples, int variant, int fallback) {
  if (g_force_op == op) return g_force_cfg;
  TuneEntry e;
  if (tune_lookup(op, kind, n, samples, variant, gpu_name(), &e)) return e.cfg;
  return fallback;
}

void tune_force(int op, int cfg) { g_force_op = op, g_force_cfg = cfg; }
void tune_release() { g_force_op = -1; }

// Times fn() with CUDA events on the stream (one warm-up run, then the faster of two runs).
template <class F>
static cudaError_t time_ms(cudaStream_t st, F fn, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  float best = 1e30f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess && rep > 0 && t < best) best = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  return e;
}

// Tries each candidate of op (run(cfg) enqueues the operation), stores and reports the fastest.
template <class R>
static purse_status tune_op(int op, int kind, int n, long long samples, int variant, const int* cands, int nc,
                            int default_cfg, cudaStream_t st, R run, purse_tune_result* out, const char* where) {
  float best = 1e30f, dms = -1.f;
  int bc = default_cfg, tried = 0;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < nc && e == cudaSuccess; ++i) {
    tune_force(op, cands[i]);
    float ms = 0.f;
    cudaError_t r = time_ms(st, [&] { return run(cands[i]); }, &ms);
    tune_release();
    if (r == cudaErrorInvalidConfiguration) {  // the shape does not fit (shared memory)
      cudaGetLastError();
      continue;
    }
    e = r;
    if (e != cudaSuccess) break;
    ++tried;
    if (cands[i] == default_cfg) dms = ms;
    if (ms < best) best = ms, bc = cands[i];
  }
  if (e != cudaSuccess) return cuda_fail(e, where);
  if (!tried) {
    set_error(std::string(where) + ": no candidate shape fits");
    return PURSE_ERR_ARG;
  }
  tune_store(op, kind, n, samples, variant, gpu_name(), TuneEntry{bc, best, dms});
  if (out) {
    out->op = op, out->config = bc, out->ms = best, out->default_config = default_cfg, out->default_ms = dms;
    out->n_tried = tried;
  }
  return PURSE_OK;
}

}  // namespace purse

using namespace purse;

extern "C" {

purse_status purse_tune_walk(purse_t h, const purse_params* p, uint64_t seed, const double* d_seeds, int s0,
                             int n_samples, void* d_q, void* d_t, purse_tune_result* out, purse_stream_t stream) {
  if (!h || !p) return (set_error("purse_tune_walk: NULL handle or params"), PURSE_ERR_ARG);
  if (n_samples < 1) return (set_error("purse_tune_walk: n_samples must be >= 1"), PURSE_ERR_ARG);
  // validate once through the real call (also the warm-up of the default shape)
  purse_status s = purse_sample(h, p, seed, d_seeds, s0, n_samples, d_q, d_t, nullptr, nullptr, stream);
  if (s != PURSE_OK) return s;
  const int cands[] = {8, 4, 2};
  cudaStream_t st = (cudaStream_t)stream;
  return tune_op(kTuneWalk, h->kind, h->n, n_samples, p->sampler + 2 * p->precision, cands, 3, 8, st,
                 [&](int) {
                   const purse_status r = purse_sample(h, p, seed, d_seeds, s0, n_samples, d_q, d_t, nullptr, nullptr,
                                                       stream);
                   if (r == PURSE_OK) return cudaSuccess;
                   return r == PURSE_ERR_ARG ? cudaErrorInvalidConfiguration : cudaErrorLaunchFailure;
                 },
                 out, "purse_tune_walk");
}

purse_status purse_tune_megb(purse_t h, int precision, int n_iters, const void* d_q, int n_rot, const void* d_t,
                             int n_tr, double* d_result, purse_tune_result* out, purse_stream_t stream) {
  if (!h) return (set_error("purse_tune_megb: NULL handle"), PURSE_ERR_ARG);
  purse_status s = megb_solve(h, precision, n_iters, d_q, n_rot, d_t, n_tr, d_result, nullptr, stream);
  if (s != PURSE_OK) return s;
  const int c64[] = {1, 2, 4, 8};
  const int c32[] = {1, 2, 4, 8, 16, 32, 64};
  const long long ns = n_rot > n_tr ? n_rot : n_tr;
  cudaStream_t st = (cudaStream_t)stream;
  return tune_op(kTuneMegb, h->kind, h->n, ns, precision, precision ? c64 : c32, precision ? 4 : 7, precision ? 1 : 4,
                 st,
                 [&](int) {
                   const purse_status r = megb_solve(h, precision, n_iters, d_q, n_rot, d_t, n_tr, d_result, nullptr,
                                                     stream);
                   return r == PURSE_OK ? cudaSuccess : cudaErrorLaunchFailure;
                 },
                 out, "purse_tune_megb");
}

purse_status purse_tune_dist(purse_t h, int mode, const float* d_poses, long long n_poses, float* d_dist,
                             purse_tune_result* out, purse_stream_t stream) {
  if (!h) return (set_error("purse_tune_dist: NULL handle"), PURSE_ERR_ARG);
  if (mode != 1 && mode != 2) return (set_error("purse_tune_dist: mode must be 1 or 2 (tensor cores)"), PURSE_ERR_ARG);
  purse_status s = purse_dist(h, mode, d_poses, n_poses, d_dist, stream);
  if (s != PURSE_OK) return s;
  const int cands[] = {2, 1};
  cudaStream_t st = (cudaStream_t)stream;
  return tune_op(kTuneDist, h->kind, h->n, n_poses, mode == 1 ? 3 : 1, cands, 2, 2, st,
                 [&](int) {
                   const purse_status r = purse_dist(h, mode, d_poses, n_poses, d_dist, stream);
                   return r == PURSE_OK ? cudaSuccess : cudaErrorLaunchFailure;
                 },
                 out, "purse_tune_dist");
}

purse_status purse_tune_cache_get(int op, int kind, int n, long long n_samples, int variant, const char* gpu,
                                  purse_tune_result* out) {
  if (!out || n < 1 || n_samples < 1) return (set_error("purse_tune_cache_get: bad argument"), PURSE_ERR_ARG);
  TuneEntry e;
  if (!tune_lookup(op, kind, n, n_samples, variant, gpu ? gpu : gpu_name(), &e)) {
    set_error("purse_tune_cache_get: no entry");
    return PURSE_ERR_STATE;
  }
  out->op = op, out->config = e.cfg, out->ms = e.ms, out->default_config = -1, out->default_ms = e.default_ms;
  out->n_tried = 0;
  return PURSE_OK;
}

purse_status purse_tune_cache_put(int op, int kind, int n, long long n_samples, int variant, const char* gpu, int config,
                                  float ms) {
  if (n < 1 || n_samples < 1 || op < 0 || op > 3) return (set_error("purse_tune_cache_put: bad argument"), PURSE_ERR_ARG);
  tune_store(op, kind, n, n_samples, variant, gpu ? gpu : gpu_name(), TuneEntry{config, ms, -1.f});
  return PURSE_OK;
}

purse_status purse_tune_cache_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.clear();
  g_tune_loaded = false;  // the file (if any) is read again at the next lookup
  return PURSE_OK;
}

}  // extern "C"
