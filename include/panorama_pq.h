/* panorama_pq.h -- IVFPQ Panorama on GB300 (sm_103a).
 *
 * Product-quantised IVF lists searched level by level with the Cauchy-Schwarz
 * bounds of Eq. 3 [Section 6.3 "IndexIVFPQPanorama"], in a basis whose level
 * energies suit product quantisation [Section 4.3 "Spectrum shaping for
 * PQ-compatibility": Procedure 1 (Robin Hood inter-level shaping),
 * Procedure 2 (intra-level isotropisation), the combined transform U R T].
 *
 * The distance an IVFPQ index ranks by is the asymmetric distance of the
 * query residual r = T(q - mu) - T(c - mu) (c the list's centroid) to a
 * vector's code: D = sum_m ||r_m - C_m[code_m]||^2 over M subvectors of
 * d / M coordinates.  The library computes it in FP32 in one fixed order:
 * each subvector term e_m = sum_j fl(fl(r_j - C_mj)^2) left to right, the
 * terms of one level added in subquantiser order, the level sums added in
 * level order.  A pruned search (mode 0) returns exactly -- bit for bit --
 * what the plain scan (mode 1) returns: a candidate is dropped only when a
 * lower bound on its computed D, with every rounding of the computation
 * accounted for, exceeds a computed D of k other candidates.
 *
 * Conventions as in panorama.h: 0 = PANO_OK, negative = error with a
 * thread-local message (panorama_last_error); caller-owned inputs and
 * outputs; library-owned index memory.
 */
#ifndef PANORAMA_PQ_H
#define PANORAMA_PQ_H

#include "panorama.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PANO_PQ 3 /* pano_index_info.precision of an IVFPQ index */

/* panorama_transform_import -- a transform from caller arrays.
 *   T:   host, d x d FP64 row-major, orthogonal (row i gives coordinate i of
 *        T(v - mu)).
 *   mu:  host, d FP64 (the centre; zeros for a pure rotation).
 *   lam: host, d FP64 >= 0, the expected variance of each output coordinate
 *        (PCA eigenvalues for a PCA basis); panorama_shape_transform reads it.
 * Errors: PANO_EINVAL (null pointer, d < 1, a non-finite value, lam < 0). */
int panorama_transform_import(const double* T, const double* mu, const double* lam, int32_t d,
                              pano_transform** out);

/* panorama_shape_transform -- U R T of Section 4.3 from a transform T whose
 * coordinates have expected variances lam (a PCA fit, or an import).
 *   n_levels: L; d % L == 0; levels are the L blocks of b = d / L coordinates.
 *   kappa:    >= 1; the cap on a level's expected energy is kappa times the
 *             mean level energy (sum lam) / L.
 *   gauss:    host, 2 d x d FP64 standard normal draws, G1 then G2
 *             (row-major).  Procedure 1: levels are visited front to back; a
 *             level whose expected energy exceeds the cap is rotated together
 *             with the smallest suffix of s >= 1 following coordinates for
 *             which b * (their summed expected variance) / (b + s) <= cap
 *             (relative tolerance 1e-12; the whole remainder if none does);
 *             the rotation of the block [a, a + n) is the Q factor, with
 *             positive diagonal R, of G1[a:a+n, a:a+n] (a Haar draw), and
 *             every coordinate of the block gets expected variance (sum) / n.
 *             Procedure 2: level l is rotated by the Q factor of G2 on its
 *             diagonal b x b block.
 *   blocks:   host, 2 * n_levels int32 or NULL: the (first coordinate, size)
 *             of each Procedure 1 rotation, then (-1, -1) entries.
 *   out:      the shaped transform (same mu; lam = the expected variances
 *             after shaping: each level's energy spread evenly).
 * Errors: PANO_EINVAL (null t / gauss / out, d % n_levels, kappa < 1 or not
 *         finite, a non-finite draw). */
int panorama_shape_transform(const pano_transform* t, int32_t n_levels, double kappa,
                             const double* gauss, int32_t* blocks, pano_transform** out);

typedef struct {
  int32_t M;             /* subquantisers: d % M == 0, M % n_levels == 0,
                            M / n_levels <= 64, d / M <= 32                   */
  int32_t n_levels;      /* L >= 1, d % L == 0 (levels of d / L coordinates)   */
  int32_t kmeans_iters;  /* coarse Lloyd iterations (default 20)               */
  int32_t pq_iters;      /* PQ Lloyd iterations (default 16)                   */
  int64_t kmeans_sample; /* coarse training rows (default min(n, 256 nlist))   */
  int64_t pq_sample;     /* PQ training rows (default min(n, 65536))           */
  uint64_t seed;         /* sampling seed (default 1234)                       */
  const float* centroids;   /* host nlist x d (original space) or NULL        */
  const int32_t* assign;    /* host n list ids in [0, nlist) or NULL = nearest
                               centroid                                       */
  const float* codebooks;   /* host M x 256 x (d / M) in the basis of t, or
                               NULL = Lloyd k-means on sampled residuals      */
  const uint8_t* codes;     /* host n x M, or NULL = nearest codeword of each
                               residual subvector (smallest FP32 term as
                               defined above, ties to the lower index)        */
} pano_pq_build_opts;

/* panorama_build_ivfpq -- an IVFPQ index of X [Section 6.3].
 *   t:      the transform (typically panorama_shape_transform's output).
 *   X:      n x d FP32 row-major, host or device.
 *   nlist:  1..n lists.  opts: required (M, n_levels).
 * Layout on the device: each list's vectors in ascending id order, in blocks
 * of 256 slots (the last one padded); per block the codes are
 * subquantiser-major, [M][256] bytes, so one level's codes for the block are
 * M / L contiguous rows of 256 bytes (the paper's sub-quantizer-major layout
 * with B = 256); per block the tail norms sqrt(||x^ tail after level l||^2)
 * [L][256] FP32 (FP64 sums from the codebook, rounded to nearest; level L-1's
 * entry is 0) and the ids [256] int32 (-1 = padding); the codebooks
 * [M][256][d / M] FP32 and the transformed centroids [nlist][d] FP32.
 * panorama_save / panorama_load keep an IVFPQ index (its quantiser arrays in
 * place of the level slices); panorama_search rejects it.
 * Errors: PANO_EINVAL (sizes above, assign or nlist out of range, fewer than
 *         256 vectors to train codebooks on), PANO_ENOMEM, PANO_ECUDA,
 *         PANO_ENODEV. */
int panorama_build_ivfpq(const pano_transform* t, const float* X, int64_t n, int32_t nlist,
                         const pano_pq_build_opts* opts, void* stream, pano_index** out);

/* panorama_search_pq -- the k smallest asymmetric distances over each query's
 * nprobe nearest lists [Section 6.3]: the query is transformed (FP32 GEMM),
 * the lists probed by original-space centroid distance (as panorama_search),
 * and each (query, list) pair is one thread block that forms the residual,
 * its level tail energies (FP64, sqrt rounded to nearest), and walks the
 * list in slabs of 2048 candidates level by level: the level's distances
 * come from a 256-entry table per subquantiser built in shared memory when
 * many candidates are live, else directly from the codebook (the same
 * arithmetic), and a candidate stops when its margined lower bound
 * (1 - gamma) * (D_head + (max(0, |s_q - s_x| - 8u (s_q + s_x)))^2) exceeds
 * the query's current k-th distance (strict).  Candidates that reach the last
 * level enter the query's top-k.  The first 64 members of each query's
 * nearest list seed the top-k before the scan.
 *   queries:  device nq x d FP32.   nprobe: 1..nlist.   k: 1..1024.
 *   out_ids / out_dists: device nq x k, ascending (distance, id), padded with
 *             (-1, +inf) when fewer than k candidates exist.
 *   mode:     0 = pruned, 1 = plain scan (every level of every candidate).
 *   collect_stats: bit 0 = count pairs, dims_scanned (coordinates whose
 *             subvector terms were added), pair_levels, reranked (candidates
 *             that reached the last level), tile_levels (tables built);
 *             bit 1 = CUDA-event times of the stages in stage_ms (transform,
 *             probe, pair order and seeds, -, verify, decode); read with
 *             panorama_search_stats.
 *   epsilon:  Eq. 4; in (0, 1) the lower bound becomes
 *             D_head + s_q^2 + s_x^2 - 2 epsilon s_q s_x (no rounding
 *             allowance): faster, approximate recall; returned distances are
 *             still the computed ones.  0 or 1 = the exact, margined test.
 * Blocks until the results are written.
 * Errors: PANO_EINVAL (not an IVFPQ index, sizes), PANO_ENOMEM, PANO_ECUDA,
 *         PANO_ENODEV, PANO_ETIMEOUT never (no device-side waits). */
int panorama_search_pq(const pano_index* idx, const float* queries, int64_t nq, int32_t nprobe,
                       int32_t k, int64_t* out_ids, float* out_dists, int32_t mode,
                       int32_t collect_stats, float epsilon, void* stream);

/* panorama_search_pq_ex -- panorama_search_pq with per-query probes and k
 * (as panorama_search_ex):
 *   nprobe:   device nq int32 (each clamped to [1, nprobe_scalar]; a
 *             nprobe_scalar < 1 means nlist), or NULL for nprobe_scalar.
 *   k:        device nq int32 (each clamped to [0, k_max]), or NULL for
 *             k_scalar in [0, k_max].
 *   k_max:    1..1024, the row length of out_ids / out_dists (nq x k_max;
 *             a row's entries past its k are (-1, +inf)).
 *   opts:     mode, collect_stats, collect_timing and epsilon are used
 *             (NULL = pruned, exact, no statistics).
 * Errors: as panorama_search_pq. */
int panorama_search_pq_ex(const pano_index* idx, const float* queries, int64_t nq,
                          const int32_t* nprobe, int32_t nprobe_scalar, const int32_t* k,
                          int32_t k_scalar, int32_t k_max, int64_t* out_ids, float* out_dists,
                          const pano_search_opts* opts, void* stream);

/* panorama_pq_export -- host copies of an IVFPQ index's quantiser.
 *   codebooks: M x 256 x (d / M) FP32, or NULL.
 *   codes:     n x M uint8 in vector-id order, or NULL.
 *   M_out:     the number of subquantisers, or NULL.
 * Errors: PANO_EINVAL (not an IVFPQ index), PANO_ECUDA. */
int panorama_pq_export(const pano_index* idx, float* codebooks, uint8_t* codes, int32_t* M_out);

/* panorama_debug_pq_encode -- the build's encoder on caller residuals: for
 * each row i and subquantiser m the codeword j with the smallest FP32 term
 * sum_t fl(fl(R[i][m dsub + t] - C[m][j][t])^2) (left to right), ties to the
 * lower j.
 *   R: device n x d FP32; codebooks: device M x 256 x (d / M) FP32;
 *   codes: device n x M uint8.  d % M == 0, d / M <= 32.
 * Errors: PANO_EINVAL, PANO_ECUDA. */
int panorama_debug_pq_encode(const float* R, int64_t n, int32_t d, int32_t M,
                             const float* codebooks, uint8_t* codes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PANORAMA_PQ_H */
