// Launchers of the BF16 / FP8 tensor-core path (verify_tc.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pano {

constexpr int TC_CHUNK = 128;  // vectors per chunk (MMA M)
constexpr int TC_QG = 64;      // queries per group (MMA N, padded to 16)
constexpr int TC_SEG = 4;      // chunks per work-item segment
// the tensor-core formats' default bound-test schedule: every chunk at the
// levels l % 4 == 0 and the last, nearly dead chunks at every level
constexpr int kTcTestEvery = 4;

struct VerifyTCArgs {
  const uint8_t* slices;
  const float* tails;
  const float* xn2;
  const float* ex;
  const int32_t* ids;
  const float* xscale;  // FP8: per-vector power-of-two scale s_x
  const float* rows;
  const int64_t* chunk_off;
  const float* qt;
  const float* qorig;
  const float4* qinfo;
  const float* qtail;
  const int32_t* kq;
  float* tau_seed;  // per-query threshold: warm start, lowered by any item
  const int4* items;
  const int* n_items;
  int* counter;
  const int32_t* bucket;
  unsigned long long* topk;
  int* err;
  unsigned long long* stats;
  int64_t items_cap;
  int d, L, max_w, k_max;
  float gslack;    // |computed - exact| terms of the bound <= gslack (|q~|+|x^|)^2
  float lb_scale;  // (1 - 8u) / (1 + eta)
  float inv_lb_up;  // 1 / lb_scale rounded up
  float ub_scale;  // (1 + 8u) / (1 - eta)
  int prune;
  // a live chunk's bound is tested at level l when l % test_every == 0, at
  // the last level, and at every level once at most 16 of its rows are live
  int test_every;
  int collect;
  int phase;  // 0: phase A (its dims are also counted apart)
  float eps;  // Eq. 4: the query tail term of the pruning test is scaled by eps
  int fp8;    // 1: E4M3 level tiles (kind::f8f6f4), 0: BF16
  int32_t level_off[65];
};

int launch_pack_bf16(const float* xt, const float* rows, const int64_t* perm, int64_t chunk0,
                     int64_t nchunks, int d, int L, const int32_t* level_off, const float* mu,
                     double c_trans, uint8_t* slices, float* tails, float* xn2, float* ex,
                     int32_t* ids, cudaStream_t st);
int launch_pack_fp8(const float* xt, const float* rows, const int64_t* perm, int64_t chunk0,
                    int64_t nchunks, int d, int L, const int32_t* level_off, const float* mu,
                    double c_trans, uint8_t* slices, float* tails, float* xn2, float* ex,
                    float* xscale, int32_t* ids, cudaStream_t st);
int launch_verify_tc(const VerifyTCArgs& a, cudaStream_t st);
size_t verify_tc_smem(int max_w, bool fp8);

}  // namespace pano
