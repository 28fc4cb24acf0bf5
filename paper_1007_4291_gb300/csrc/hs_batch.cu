// Batching around the sweep: applications of several plans as one CUDA graph
// whose per-problem stage chains run concurrently, and the chunk-length
// autotuner with its text cache.
//
// The stage chain of one problem is strictly sequential (Algorithm 4: each
// block needs the previous block's result), so a small problem (n = 255 has
// 9 stages of 8 chunks per front) occupies a few SMs for a few hundred
// microseconds.  Independent problems are the natural source of parallelism:
// the batched application forks one branch per problem inside a single
// captured graph, and the runtime executes the branches side by side.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include "hs_internal.cuh"

namespace hs {
namespace {

struct BatchEntry {
  std::vector<long long> key;   // (uid, r, z, nrhs) per problem, then dtype
  std::vector<long long> uids;
  cudaGraphExec_t exec;
  long long kernels;
};

std::mutex g_batch_mutex;
std::vector<BatchEntry> g_batch;    // most recently used last
constexpr size_t kMaxBatchGraphs = 16;

void drop_entry(size_t i) {
  cudaGraphExecDestroy(g_batch[i].exec);
  g_batch.erase(g_batch.begin() + (long)i);
}

}  // namespace

void forget_batch_graphs(long long uid) {
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  for (size_t i = g_batch.size(); i-- > 0;) {
    const auto& u = g_batch[i].uids;
    if (std::find(u.begin(), u.end(), uid) != u.end()) drop_entry(i);
  }
}

// Chunk length (and separator grouping, 0 when the entry has none) recorded
// by hs_autotune for this key, or 0.
int tuned_chunk(const char* path, int n, int bp, int b, int dL, int prec, int nrhs, int* sep) {
  *sep = 0;
  if (!path) return 0;
  FILE* f = std::fopen(path, "r");
  if (!f) return 0;
  char line[256];
  int best = 0;
  while (std::fgets(line, sizeof(line), f)) {
    int kn, kbp, kb, kdl, kp, kr, chunk, ks = 0;
    double ms;
    const int got = std::sscanf(line, "2d n=%d bp=%d b=%d d=%d prec=%d nrhs=%d chunk=%d sep=%d ms=%lf", &kn, &kbp,
                                &kb, &kdl, &kp, &kr, &chunk, &ks, &ms);
    if (got != 9) {     // entries without a separator grouping
      ks = 0;
      if (std::sscanf(line, "2d n=%d bp=%d b=%d d=%d prec=%d nrhs=%d chunk=%d ms=%lf", &kn, &kbp, &kb, &kdl, &kp,
                      &kr, &chunk, &ms) != 8)
        continue;
    }
    if (kn == n && kbp == bp && kb == b && kdl == dL && kp == prec && kr == nrhs && chunk >= 2 &&
        (ks == 0 || ks == 1 || ks == 2 || ks == 4)) {
      best = chunk;  // the last entry for a key wins
      *sep = ks;
    }
  }
  std::fclose(f);
  return best;
}

}  // namespace hs

using namespace hs;

extern "C" int hs_apply_batched(int nprob, hs_plan* const* plans, const void* const* r, void* const* z,
                                const int* nrhs, int dtype, void* stream) {
  if (nprob < 1 || !plans || !r || !z || !nrhs || (dtype != HS_C64 && dtype != HS_C128)) return HS_EINVAL;
  std::vector<Plan*> ps(nprob);
  std::vector<long long> key, uids;
  for (int k = 0; k < nprob; ++k) {
    if (!plans[k] || !r[k] || !z[k]) return HS_EINVAL;
    ps[k] = reinterpret_cast<Plan*>(plans[k]);
    if (nrhs[k] < 1 || nrhs[k] > ps[k]->max_nrhs) return HS_EINVAL;
    if (std::find(uids.begin(), uids.end(), ps[k]->uid) != uids.end()) return HS_EINVAL;
    uids.push_back(ps[k]->uid);
    key.insert(key.end(), {ps[k]->uid, (long long)(uintptr_t)r[k], (long long)(uintptr_t)z[k], (long long)nrhs[k]});
  }
  key.push_back(dtype);
  cudaStream_t s = (cudaStream_t)stream;
  for (Plan* q : ps) plan_wait(*q, s);
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  for (size_t i = 0; i < g_batch.size(); ++i) {
    if (g_batch[i].key == key) {
      BatchEntry e = g_batch[i];
      g_batch.erase(g_batch.begin() + (long)i);
      g_batch.push_back(e);
      note_launch(e.kernels);
      cudaError_t ce = cudaGraphLaunch(e.exec, s);
      return ce == cudaSuccess ? HS_OK : cuda_status(ce);
    }
  }
  sweep_prepare_attributes(HS_C64);
  sweep_prepare_attributes(HS_C128);
  // capture: fork one branch per problem from the origin stream, join at the end
  std::vector<cudaStream_t> br(nprob, nullptr);
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  int st = HS_OK;
  auto cleanup = [&]() {
    for (auto q : br) if (q) cudaStreamDestroy(q);
    if (origin) cudaStreamDestroy(origin);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
  };
  if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
    cleanup();
    return HS_ECUDA;
  }
  for (int k = 0; k < nprob; ++k)
    if (cudaStreamCreateWithFlags(&br[k], cudaStreamNonBlocking) != cudaSuccess) { cleanup(); return HS_ECUDA; }
  BatchEntry e{};
  e.key = key;
  e.uids = uids;
  st = capture_graph(origin, [&](cudaStream_t c) -> int {
    if (cudaEventRecord(fork, c) != cudaSuccess) return HS_ECUDA;
    for (int k = 0; k < nprob; ++k) {
      Plan& p = *ps[k];
      if (cudaStreamWaitEvent(br[k], fork, 0) != cudaSuccess) return HS_ECUDA;
      const int n2 = p.n * p.n;
      int s2 = layout_to_internal(r[k], dtype, p.d_u, p.prec, n2, nrhs[k], br[k]);
      if (s2 == HS_OK) s2 = sweep_launch(p, nrhs[k], br[k]);
      if (s2 == HS_OK) s2 = layout_from_internal(p.d_u, p.prec, z[k], dtype, n2, nrhs[k], br[k]);
      if (s2 != HS_OK) return s2;
      if (cudaEventRecord(join, br[k]) != cudaSuccess || cudaStreamWaitEvent(c, join, 0) != cudaSuccess)
        return HS_ECUDA;
    }
    return HS_OK;
  }, &e.exec, &e.kernels);
  cleanup();
  if (st != HS_OK) return st;
  if (g_batch.size() >= kMaxBatchGraphs) drop_entry(0);
  g_batch.push_back(e);
  note_launch(e.kernels);
  cudaError_t ce = cudaGraphLaunch(e.exec, s);
  return ce == cudaSuccess ? HS_OK : cuda_status(ce);
}

extern "C" int hs_autotune(const double* c, double omega, int n, int dim, int pml_width, int moving_pml_width,
                           const hs_options* opt_in, int nrhs, void* stream, int* best_chunk, double* best_ms,
                           int* best_sep) {
  if (!best_chunk || nrhs < 1) return HS_EINVAL;
  if (dim != 2) return HS_EUNSUPPORTED;
  *best_chunk = 0;
  int bsep = 0;
  hs_options opt;
  hs_default_options(&opt);
  if (opt_in) opt = *opt_in;
  opt.max_nrhs = nrhs;
  opt.tune_cache = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  const int lmin = 2;
  std::vector<int> cand;
  int dev = 0, sms = 2;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // lengths that give one chunk CTA per pair of SMs (one full wave), per SM,
  // and a set of fixed lengths (setup raises a length that needs too many
  // separators)
  for (int per_front : {std::max(1, sms / 2), std::max(1, sms), std::max(1, sms / 4)}) {
    const int L = std::max(lmin, (n + per_front - 1) / per_front);
    if (L <= n && std::find(cand.begin(), cand.end(), L) == cand.end()) cand.push_back(L);
  }
  for (int L : {8, 12, 16, 24, 32, 48, 64, 96, 128})
    if (L >= lmin && L <= n && std::find(cand.begin(), cand.end(), L) == cand.end()) cand.push_back(L);
  if (cand.empty()) cand.push_back(std::min(n, std::max(lmin, 2)));
  const size_t bytes = (size_t)n * n * nrhs * (opt.factor_prec == HS_C64 ? 8 : 16);
  void* buf = nullptr;
  HS_CUDA_TRY(cudaMalloc(&buf, bytes));
  cudaMemsetAsync(buf, 0, bytes, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e300;
  int st = HS_OK;
  for (int L : cand) {
    opt.chunk = L;
    hs_plan* plan = nullptr;
    int s2 = hs_setup(c, omega, n, dim, pml_width, moving_pml_width, &opt, stream, &plan);
    if (s2 == HS_EUNSUPPORTED) continue;  // e.g. separator chain too long for this length
    if (s2 != HS_OK) { st = s2; break; }
    const int dtype = opt.factor_prec;
    Plan& pp = *reinterpret_cast<Plan*>(plan);
    for (int sep : {1, 2, 4}) {
      // a new grouping changes the launches: the sweep graph is captured anew
      cudaStreamSynchronize(s);
      release_sweep_graphs(pp);
      pp.opt.sep_rhs_per_cta = sep;
      s2 = hs_apply(plan, buf, buf, nrhs, dtype, stream);  // warm-up (and graph capture)
      const int reps = 3;
      cudaEventRecord(e0, s);
      for (int k = 0; k < reps && s2 == HS_OK; ++k) s2 = hs_apply(plan, buf, buf, nrhs, dtype, stream);
      cudaEventRecord(e1, s);
      cudaError_t ce = cudaEventSynchronize(e1);
      if (s2 == HS_OK && ce != cudaSuccess) s2 = cuda_status(ce);
      if (s2 == HS_OK) s2 = hs_last_device_status(plan);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (s2 == HS_EUNSUPPORTED) { s2 = HS_OK; continue; }  // this length and grouping do not fit
      if (s2 != HS_OK) break;
      if (ms / reps < best) { best = ms / reps; *best_chunk = L; bsep = sep; }
    }
    hs_destroy(plan);
    if (s2 != HS_OK) { st = s2; break; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (st != HS_OK) return st;
  if (*best_chunk == 0) return HS_EUNSUPPORTED;
  if (best_ms) *best_ms = best;
  if (best_sep) *best_sep = bsep;
  if (opt_in && opt_in->tune_cache) {
    FILE* f = std::fopen(opt_in->tune_cache, "a");
    if (!f) return HS_EINVAL;
    std::fprintf(f, "2d n=%d bp=%d b=%d d=%d prec=%d nrhs=%d chunk=%d sep=%d ms=%.4f\n", n, pml_width,
                 moving_pml_width, opt.layers_per_step, opt.factor_prec, nrhs, *best_chunk, bsep, best);
    std::fclose(f);
  }
  return HS_OK;
}
