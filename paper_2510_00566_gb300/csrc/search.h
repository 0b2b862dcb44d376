// Host entry points of the search path (see search.cu).
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace pano {
int search(const pano_index* ip, const float* queries, int64_t nq, const int32_t* nprobe,
           int32_t nprobe_scalar, const int32_t* k, int32_t k_scalar, int32_t k_max,
           int64_t* out_ids, float* out_dists, cudaStream_t st, const pano_search_opts* opts,
           void* ext_ws = nullptr, size_t ext_cap = 0, int* err_host = nullptr);
// Bytes of the device workspace one search of nq queries (probe stride
// `stride`, k_max results) carves, as search() computes it.
int search_workspace_bytes(const pano_index* ip, int64_t nq, int32_t stride, int32_t k_max,
                           size_t* out);
// Status code of a device error word (kErrTimeout -> PANO_ETIMEOUT,
// kErrBadInput -> PANO_EINVAL, otherwise PANO_OK).
int status_of_device_error(int word);
int probe_only(const pano_index* ip, const float* queries, int64_t nq, int32_t nprobe,
               int32_t* out, cudaStream_t st);
const pano_search_stats& last_stats();
pano_search_stats& stats_slot();  // the calling thread's last-call statistics
int transform_queries(const pano_index& I, const float* queries, int64_t nq, float* qt,
                      float4* qinfo, float* qtail, float* qn2, cudaStream_t st);
int build_flat(const pano_transform* t, const float* X, int64_t n, const pano_build_opts* o,
               cudaStream_t st, pano_index** out);
int refine(const pano_index* ip, const float* queries, int64_t nq, const int64_t* cand,
           int32_t kprime, int32_t k, int64_t* out_ids, float* out_dists, float epsilon,
           cudaStream_t st);
int build_ivf(const pano_transform* t, const float* X, int64_t n, int nlist,
              const pano_build_opts* o, cudaStream_t st, pano_index** out);
int make_levels(int d, const pano_build_opts* o, std::vector<int32_t>& widths,
                std::vector<int32_t>& offs);
int check_device(int* dev_out);
int coarse_lists(const float* Xd, int64_t n, int d, int nlist, const pano_build_opts* o,
                 cudaStream_t st, pano_index& I);
}  // namespace pano
