/* Brute-force answer of Problem 1 over IVF candidate sets, FP64, plain C.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the CUDA library never
 * links or calls this file, and this file includes none of the library's
 * headers.
 *
 * For query i the candidate set Gamma(i) is the union of the lists
 * probes[i][0 .. nprobe[i]) (Problem 2 with an IVF index, Section 6.1); list c
 * holds database rows rows[ptr[c] .. ptr[c+1]).  Every candidate's squared
 * distance is sum_j (q_j - x_j)^2 accumulated in double from the FP32 inputs
 * (Problem 1).  The k smallest (dist, id) pairs are returned in ascending
 * order, ties broken by id, padded with (-1, +inf) when |Gamma| < k.
 * Queries are split across `nthreads` POSIX threads.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
  const float* X;
  int32_t d;
  const float* Q;
  const int64_t* ptr;
  const int64_t* rows;
  const int32_t* probes;
  int32_t probe_stride;
  const int32_t* nprobe;
  const int32_t* k;
  int32_t k_max;
  int64_t* out_ids;
  double* out_d;
  int64_t q_begin, q_end;
} job_t;

/* (da, ia) before (db, ib) in the (dist, id) order */
static int before(double da, int64_t ia, double db, int64_t ib) {
  return da < db || (da == db && ia < ib);
}

static void* run(void* arg) {
  job_t* j = (job_t*)arg;
  for (int64_t i = j->q_begin; i < j->q_end; ++i) {
    const float* q = j->Q + i * (int64_t)j->d;
    int k = j->k[i];
    double* bd = j->out_d + i * (int64_t)j->k_max;
    int64_t* bi = j->out_ids + i * (int64_t)j->k_max;
    for (int t = 0; t < j->k_max; ++t) {
      bd[t] = INFINITY;
      bi[t] = -1;
    }
    int filled = 0;
    for (int p = 0; p < j->nprobe[i]; ++p) {
      int32_t c = j->probes[i * (int64_t)j->probe_stride + p];
      for (int64_t r = j->ptr[c]; r < j->ptr[c + 1]; ++r) {
        int64_t row = j->rows[r];
        const float* x = j->X + row * (int64_t)j->d;
        double s = 0.0;
        for (int32_t t = 0; t < j->d; ++t) {
          double diff = (double)q[t] - (double)x[t];
          s += diff * diff;
        }
        /* insertion into the sorted k-best array */
        if (filled < k) {
          int pos = filled++;
          while (pos > 0 && before(s, row, bd[pos - 1], bi[pos - 1])) {
            bd[pos] = bd[pos - 1];
            bi[pos] = bi[pos - 1];
            --pos;
          }
          bd[pos] = s;
          bi[pos] = row;
        } else if (k > 0 && before(s, row, bd[k - 1], bi[k - 1])) {
          int pos = k - 1;
          while (pos > 0 && before(s, row, bd[pos - 1], bi[pos - 1])) {
            bd[pos] = bd[pos - 1];
            bi[pos] = bi[pos - 1];
            --pos;
          }
          bd[pos] = s;
          bi[pos] = row;
        }
      }
    }
  }
  return NULL;
}

int oracle_ivf_topk(const float* X, int32_t d, const float* Q, int64_t nq,
                    const int64_t* ptr, const int64_t* rows,
                    const int32_t* probes, int32_t probe_stride,
                    const int32_t* nprobe, const int32_t* k, int32_t k_max,
                    int64_t* out_ids, double* out_d, int32_t nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > nq) nthreads = nq > 0 ? (int32_t)nq : 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
  job_t* jobs = (job_t*)malloc(sizeof(job_t) * nthreads);
  if (!th || !jobs) {
    free(th);
    free(jobs);
    return -1;
  }
  int64_t per = (nq + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    job_t j = {X, d, Q, ptr, rows, probes, probe_stride, nprobe, k, k_max,
               out_ids, out_d, t * per, (t + 1) * per};
    if (j.q_begin > nq) j.q_begin = nq;
    if (j.q_end > nq) j.q_end = nq;
    jobs[t] = j;
    pthread_create(&th[t], NULL, run, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
  return 0;
}
