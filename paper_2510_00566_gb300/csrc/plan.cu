// Search plans (a batch of fixed shape captured into one CUDA graph) and the
// autotuners (level split; storage precision x level split).
//
// A plan records every step of one search -- workspace allocation, memsets,
// the transform / probe GEMMs, work inversion, the two persistent verify
// kernels and the decode -- on a private stream under thread-local capture
// and instantiates the graph; launching the plan replays all of it with one
// cudaGraphLaunch.  The device pointers given at creation are baked into the
// graph: each launch reads their current contents.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "search.h"

struct pano_plan {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = 0;
  ~pano_plan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

using namespace pano;

extern "C" {

int panorama_plan_create(const pano_index* idx, const float* queries, int64_t nq,
                         const int32_t* nprobe, int32_t nprobe_scalar, const int32_t* k,
                         int32_t k_scalar, int32_t k_max, int64_t* out_ids, float* out_dists,
                         int32_t mode, pano_plan** out) {
  pano_search_opts o{};
  o.mode = mode;
  return panorama_plan_create_ex(idx, queries, nq, nprobe, nprobe_scalar, k, k_scalar, k_max,
                                 out_ids, out_dists, &o, out);
}

int panorama_plan_create_ex(const pano_index* idx, const float* queries, int64_t nq,
                            const int32_t* nprobe, int32_t nprobe_scalar, const int32_t* k,
                            int32_t k_scalar, int32_t k_max, int64_t* out_ids, float* out_dists,
                            const pano_search_opts* opts, pano_plan** out) {
  clear_error();
  PANO_CHECK(idx && out && nq >= 1, PANO_EINVAL, "bad arguments to plan_create");
  auto plan = std::make_unique<pano_plan>();
  PANO_CUDA(cudaGetDevice(&plan->device));
  cudaStream_t cs = nullptr;
  PANO_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  // kernel attributes and occupancy are settled by one eager search first
  pano_search_opts o{};
  if (opts) o = *opts;
  o.collect_stats = 0;
  o.collect_timing = 0;
  o.synchronize = 1;
  int rc = search(idx, queries, nq, nprobe, nprobe_scalar, k, k_scalar, k_max, out_ids,
                  out_dists, cs, &o);
  if (rc) {
    cudaStreamDestroy(cs);
    return rc;
  }
  o.synchronize = 0;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  rc = search(idx, queries, nq, nprobe, nprobe_scalar, k, k_scalar, k_max, out_ids, out_dists,
              cs, &o);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  plan->graph = g;
  PANO_CUDA(cudaGraphInstantiate(&plan->exec, g, 0));
  *out = plan.release();
  return PANO_OK;
}

int panorama_plan_launch(pano_plan* plan, void* stream) {
  clear_error();
  PANO_CHECK(plan && plan->exec, PANO_EINVAL, "null plan");
  PANO_CUDA(cudaGraphLaunch(plan->exec, (cudaStream_t)stream));
  return PANO_OK;
}

void panorama_plan_free(pano_plan* plan) { delete plan; }

int panorama_autotune_levels(const pano_transform* t, const float* X, int64_t n,
                             const float* queries, int64_t nq, int32_t nlist, int32_t nprobe,
                             int32_t k, int32_t precision, const int32_t* widths,
                             const int32_t* n_levels, int32_t n_candidates, int32_t repeats,
                             int32_t* best, float* ms_out, void* stream) {
  clear_error();
  PANO_CHECK(t && X && queries && widths && n_levels && best && n_candidates >= 1 && nq >= 1 &&
                 nlist >= 1 && nprobe >= 1 && nprobe <= nlist && k >= 1,
             PANO_EINVAL, "bad arguments to autotune_levels");
  cudaStream_t st = (cudaStream_t)stream;
  repeats = std::max(1, repeats);
  const int d = t->d;
  int64_t* ids = nullptr;
  float* dists = nullptr;
  PANO_CUDA(cudaMalloc(&ids, (size_t)nq * k * 8));
  PANO_CUDA(cudaMalloc(&dists, (size_t)nq * k * 4));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<float> cent;  // k-means once, shared by every candidate
  int rc = PANO_OK;
  float best_ms = INFINITY;
  *best = -1;
  const int32_t* wp = widths;
  for (int c = 0; c < n_candidates && rc == PANO_OK; ++c) {
    pano_build_opts o{};
    o.n_levels = n_levels[c];
    o.level_widths = wp;
    o.precision = precision;
    o.seed = 1234;
    if (!cent.empty()) o.centroids = cent.data();
    wp += n_levels[c];
    pano_index* idx = nullptr;
    int brc = build_ivf(t, X, n, nlist, &o, st, &idx);
    if (brc) {  // an unsupported split is skipped, not fatal
      if (ms_out) ms_out[c] = INFINITY;
      continue;
    }
    if (cent.empty()) cent = idx->centroids;
    std::vector<float> times;
    for (int r = 0; r <= repeats && rc == PANO_OK; ++r) {
      cudaEventRecord(e0, st);
      rc = search(idx, queries, nq, nullptr, nprobe, nullptr, k, k, ids, dists, st, nullptr);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) times.push_back(ms);  // the first search warms up
    }
    delete idx;
    if (rc) break;
    std::sort(times.begin(), times.end());
    const float med = times[times.size() / 2];
    if (ms_out) ms_out[c] = med;
    if (med < best_ms) {
      best_ms = med;
      *best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(ids);
  cudaFree(dists);
  if (rc) return rc;
  PANO_CHECK(*best >= 0, PANO_EINVAL, "no candidate level split could be built");
  (void)d;
  return PANO_OK;
}

namespace {

// Widths a storage format's verify kernels take (BF16: 16, 32 or 64 / 128,
// FP8: 32, 64, 128 or 256 -- the swizzled tile layouts and what fits in
// shared memory; FP32: multiples of 4 up to 256).
bool width_ok(int w, int precision) {
  if (precision == PANO_BF16) return w == 16 || w == 32 || w == 64 || w == 128;
  if (precision == PANO_FP8) return w == 32 || w == 64 || w == 128 || w == 256;
  return w >= 4 && w % 4 == 0 && w <= 256;
}

// Candidate level splits of d for one storage format: every uniform width
// that divides d, and front-loaded splits whose leading levels are narrow
// (most candidates are pruned there) and double towards the widest the
// format takes, the last level taking what is left.
std::vector<std::vector<int32_t>> candidate_splits(int d, int precision) {
  std::vector<std::vector<int32_t>> out;
  const int maxw = precision == PANO_BF16 ? 128 : 256;
  for (int w : {16, 32, 64, 128, 256})
    if (d % w == 0 && width_ok(w, precision) && d / w <= 64 && d / w >= 1)
      out.push_back(std::vector<int32_t>(d / w, w));
  for (int w0 : {16, 32, 64}) {
    std::vector<int32_t> v;
    int sum = 0, w = w0;
    bool ok = true;
    while (sum < d && ok) {
      int take = std::min(w, d - sum);
      ok = width_ok(take, precision);
      v.push_back(take);
      sum += take;
      w = std::min(2 * w, maxw);
    }
    if (ok && v.size() <= 64 && v.size() > 1 &&
        std::find(out.begin(), out.end(), v) == out.end())
      out.push_back(v);
  }
  return out;
}

}  // namespace

int panorama_autotune(const pano_transform* t, const float* X, int64_t n, const float* queries,
                      int64_t nq, int32_t nlist, int32_t nprobe, int32_t k,
                      const int32_t* precisions, int32_t n_prec, const int32_t* widths,
                      const int32_t* n_levels, int32_t n_candidates, int32_t repeats,
                      pano_autotune_trial* trials, int32_t max_trials, int32_t* n_trials,
                      int32_t* best, void* stream) {
  clear_error();
  PANO_CHECK(t && X && queries && precisions && n_prec >= 1 && trials && max_trials >= 1 &&
                 n_trials && best && nq >= 1 && nlist >= 1 && nprobe >= 1 && nprobe <= nlist &&
                 k >= 1 && k <= 1024,
             PANO_EINVAL, "bad arguments to autotune");
  PANO_CHECK(!n_candidates || (widths && n_levels), PANO_EINVAL, "candidate widths missing");
  for (int i = 0; i < n_prec; ++i)
    PANO_CHECK(precisions[i] == PANO_FP32 || precisions[i] == PANO_BF16 ||
                   precisions[i] == PANO_FP8,
               PANO_EINVAL, "autotune precisions are FP32, BF16 or FP8");
  cudaStream_t st = (cudaStream_t)stream;
  repeats = std::max(1, repeats);
  const int d = t->d;
  // the (precision, split) pairs, precision-major
  std::vector<std::pair<int, std::vector<int32_t>>> pairs;
  for (int i = 0; i < n_prec; ++i) {
    if (n_candidates > 0) {
      const int32_t* wp = widths;
      for (int c = 0; c < n_candidates; ++c) {
        PANO_CHECK(n_levels[c] >= 1 && n_levels[c] <= 64, PANO_EINVAL, "1..64 levels");
        pairs.emplace_back(precisions[i], std::vector<int32_t>(wp, wp + n_levels[c]));
        wp += n_levels[c];
      }
    } else {
      for (auto& v : candidate_splits(d, precisions[i])) pairs.emplace_back(precisions[i], v);
    }
  }
  PANO_CHECK(!pairs.empty(), PANO_EINVAL, "no candidate level split for this dimension");
  PANO_CHECK((int64_t)pairs.size() <= max_trials, PANO_EINVAL,
             "more candidates (" + std::to_string(pairs.size()) + ") than max_trials");
  int64_t* ids = nullptr;
  float* dists = nullptr;
  PANO_CUDA(cudaMalloc(&ids, (size_t)nq * k * 8));
  PANO_CUDA(cudaMalloc(&dists, (size_t)nq * k * 4));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<float> cent;  // k-means once, shared by every candidate
  int rc = PANO_OK;
  float best_ms = INFINITY;
  *best = -1;
  *n_trials = 0;
  for (size_t c = 0; c < pairs.size() && rc == PANO_OK; ++c) {
    pano_autotune_trial& tr = trials[c];
    std::memset(&tr, 0, sizeof(tr));
    tr.precision = pairs[c].first;
    tr.n_levels = (int32_t)pairs[c].second.size();
    std::copy(pairs[c].second.begin(), pairs[c].second.end(), tr.widths);
    tr.ms = INFINITY;
    ++*n_trials;
    pano_build_opts o{};
    o.n_levels = tr.n_levels;
    o.level_widths = tr.widths;
    o.precision = tr.precision;
    o.seed = 1234;
    if (!cent.empty()) o.centroids = cent.data();
    pano_index* idx = nullptr;
    if (build_ivf(t, X, n, nlist, &o, st, &idx)) continue;  // not buildable: +inf
    if (cent.empty()) cent = idx->centroids;
    // the bound-test schedules: every level (Algorithm 1), every other,
    // every fourth, the first and last levels only (the tensor-core formats
    // also test nearly dead chunks at every level)
    std::vector<uint64_t> seen;  // tested-level masks already timed
    for (int te : {1, 2, 4, (int)tr.n_levels}) {
      uint64_t mask = 1ull << (tr.n_levels - 1);
      for (int l = 0; l < tr.n_levels; ++l)
        if (l % te == 0) mask |= 1ull << l;
      if (std::find(seen.begin(), seen.end(), mask) != seen.end()) continue;
      seen.push_back(mask);
      pano_search_opts so{};
      so.synchronize = 1;
      so.test_every = te;
      std::vector<float> times;
      for (int r = 0; r <= repeats && rc == PANO_OK; ++r) {
        cudaEventRecord(e0, st);
        rc = search(idx, queries, nq, nullptr, nprobe, nullptr, k, k, ids, dists, st, &so);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) times.push_back(ms);  // the first search warms up
      }
      if (rc) break;
      std::sort(times.begin(), times.end());
      if (times[times.size() / 2] < tr.ms) {
        tr.ms = times[times.size() / 2];
        tr.test_every = te;
      }
    }
    delete idx;
    if (rc == PANO_EINVAL) {  // a split the search cannot stage: not a candidate
      rc = PANO_OK;
      clear_error();
      tr.ms = INFINITY;
      tr.test_every = 0;
      continue;
    }
    if (rc) break;
    if (tr.ms < best_ms) {
      best_ms = tr.ms;
      *best = (int32_t)c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(ids);
  cudaFree(dists);
  if (rc) return rc;
  PANO_CHECK(*best >= 0, PANO_EINVAL, "no candidate could be built and searched");
  return PANO_OK;
}

}  // extern "C"
