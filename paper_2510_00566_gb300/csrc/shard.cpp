// Host-side helpers of a search sharded by IVF lists (see panorama.h):
// balanced list ownership and the exact k-way merge of per-shard top-k.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <unordered_set>
#include <vector>

#include "internal.h"

using namespace pano;

extern "C" {

int panorama_partition_lists(const int32_t* list_size, int32_t nlist, int32_t n_shards,
                             int32_t* owner) {
  clear_error();
  PANO_CHECK(list_size && owner && nlist >= 1 && n_shards >= 1, PANO_EINVAL,
             "bad arguments to partition_lists");
  for (int32_t c = 0; c < nlist; ++c)
    PANO_CHECK(list_size[c] >= 0, PANO_EINVAL, "negative list size");
  std::vector<int32_t> order(nlist);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return list_size[a] > list_size[b]; });
  std::vector<int64_t> load(n_shards, 0);
  for (int32_t c : order) {
    int32_t best = 0;
    for (int32_t s = 1; s < n_shards; ++s)
      if (load[s] < load[best]) best = s;
    owner[c] = best;
    load[best] += list_size[c];
  }
  return PANO_OK;
}

int panorama_merge_topk(const int64_t* ids, const float* dists, int32_t n_parts, int64_t nq,
                        int32_t k, int64_t* out_ids, float* out_dists) {
  clear_error();
  PANO_CHECK(n_parts >= 1 && nq >= 0 && k >= 1, PANO_EINVAL, "bad arguments to merge_topk");
  if (nq == 0) return PANO_OK;
  PANO_CHECK(ids && dists && out_ids && out_dists, PANO_EINVAL, "null argument to merge_topk");
  struct Key {
    float d;
    int64_t id;
  };
  std::vector<Key> all;
  all.reserve((size_t)n_parts * k);
  std::unordered_set<int64_t> seen;
  for (int64_t i = 0; i < nq; ++i) {
    all.clear();
    for (int32_t p = 0; p < n_parts; ++p) {
      const int64_t* ri = ids + ((int64_t)p * nq + i) * k;
      const float* rd = dists + ((int64_t)p * nq + i) * k;
      for (int32_t j = 0; j < k; ++j)
        if (ri[j] >= 0) all.push_back({rd[j], ri[j]});
    }
    std::sort(all.begin(), all.end(), [](const Key& a, const Key& b) {
      return a.d < b.d || (a.d == b.d && a.id < b.id);
    });
    seen.clear();
    int32_t j = 0;
    for (size_t e = 0; e < all.size() && j < k; ++e)
      if (seen.insert(all[e].id).second) {  // first (smallest) occurrence of an id
        out_ids[i * k + j] = all[e].id;
        out_dists[i * k + j] = all[e].d;
        ++j;
      }
    for (; j < k; ++j) {
      out_ids[i * k + j] = -1;
      out_dists[i * k + j] = INFINITY;
    }
  }
  return PANO_OK;
}

}  // extern "C"
