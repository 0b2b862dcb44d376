// Search plans (a batch of fixed shape captured into one CUDA graph) and the
// level-width autotuner.
//
// A plan records every step of one search -- workspace allocation, memsets,
// the transform / probe GEMMs, work inversion, the two persistent verify
// kernels and the decode -- on a private stream under thread-local capture
// and instantiates the graph; launching the plan replays all of it with one
// cudaGraphLaunch.  The device pointers given at creation are baked into the
// graph: each launch reads their current contents.
#include <algorithm>
#include <cmath>
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
  clear_error();
  PANO_CHECK(idx && out && nq >= 1, PANO_EINVAL, "bad arguments to plan_create");
  auto plan = std::make_unique<pano_plan>();
  PANO_CUDA(cudaGetDevice(&plan->device));
  cudaStream_t cs = nullptr;
  PANO_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  // kernel attributes and occupancy are settled by one eager search first
  pano_search_opts o{};
  o.mode = mode;
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

}  // extern "C"
