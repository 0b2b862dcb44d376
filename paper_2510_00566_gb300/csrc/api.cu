// C-ABI of the library (declared in include/panorama.h): argument checks,
// error reporting, the host PCA fit, index inspection and persistence.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>

#include "../../include/panorama_pq.h"
#include "internal.h"
#include "search.h"

namespace pano {

static thread_local std::string t_err;

void set_error(const std::string& msg) { t_err = msg; }
void clear_error() { t_err.clear(); }
int fail(int code, const std::string& msg) {
  t_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  t_err = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return PANO_ENOMEM;
  return PANO_ECUDA;
}

namespace {

// --------------------------------------------------------------- file I/O
constexpr char kMagic[8] = {'P', 'A', 'N', 'O', 'I', 'D', 'X', '1'};
constexpr uint32_t kVersion = 1;

struct Fnv {
  uint64_t h = 0xcbf29ce484222325ULL;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 0x100000001b3ULL;
    }
  }
};

struct Writer {
  std::ofstream f;
  Fnv fnv;
  bool ok = true;
  void raw(const void* p, size_t n) {
    if (!ok) return;
    f.write(static_cast<const char*>(p), (std::streamsize)n);
    fnv.add(p, n);
    ok = (bool)f;
  }
  template <class T>
  void pod(const T& v) { raw(&v, sizeof(T)); }
  template <class T>
  void vec(const std::vector<T>& v) {
    uint64_t n = v.size();
    pod(n);
    raw(v.data(), n * sizeof(T));
  }
  int dev(const DevBuf& b) {
    uint64_t n = b.bytes;
    pod(n);
    std::vector<char> tmp(std::min<uint64_t>(n, 64ull << 20));
    for (uint64_t o = 0; o < n; o += tmp.size()) {
      size_t m = (size_t)std::min<uint64_t>(tmp.size(), n - o);
      PANO_CUDA(cudaMemcpy(tmp.data(), (char*)b.p + o, m, cudaMemcpyDeviceToHost));
      raw(tmp.data(), m);
    }
    return PANO_OK;
  }
};

struct Reader {
  std::ifstream f;
  Fnv fnv;
  bool ok = true;
  uint64_t remaining = 0;  // bytes left before the checksum
  void raw(void* p, size_t n) {
    if (!ok || n > remaining) {
      ok = false;
      return;
    }
    f.read(static_cast<char*>(p), (std::streamsize)n);
    ok = (bool)f;
    if (ok) fnv.add(p, n);
    remaining -= n;
  }
  template <class T>
  void pod(T& v) { raw(&v, sizeof(T)); }
  template <class T>
  void vec(std::vector<T>& v, uint64_t max_n) {
    uint64_t n = 0;
    pod(n);
    if (!ok || n > max_n || n * sizeof(T) > remaining) {
      ok = false;
      return;
    }
    v.resize(n);
    raw(v.data(), n * sizeof(T));
  }
  int dev(DevBuf& b, uint64_t expect) {
    uint64_t n = 0;
    pod(n);
    if (!ok || n != expect || n > remaining) {
      ok = false;
      return PANO_OK;
    }
    int rc = b.alloc(n);
    if (rc) return rc;
    std::vector<char> tmp(std::min<uint64_t>(std::max<uint64_t>(n, 1), 64ull << 20));
    for (uint64_t o = 0; o < n && ok; o += tmp.size()) {
      size_t m = (size_t)std::min<uint64_t>(tmp.size(), n - o);
      raw(tmp.data(), m);
      if (!ok) break;
      PANO_CUDA(cudaMemcpy((char*)b.p + o, tmp.data(), m, cudaMemcpyHostToDevice));
    }
    return PANO_OK;
  }
};

}  // namespace
}  // namespace pano

using namespace pano;

extern "C" {

const char* panorama_last_error(void) { return t_err.c_str(); }
const char* panorama_version(void) { return "panorama-gb300 0.1 (sm_103a)"; }

int panorama_fit_transform(const float* X, int64_t n, int32_t d, const pano_build_opts* opts,
                           pano_transform** out) {
  clear_error();
  PANO_CHECK(X && out && n >= 1 && d >= 1, PANO_EINVAL, "bad arguments to fit_transform");
  auto t = std::make_unique<pano_transform>();
  t->d = d;
  t->identity = opts ? opts->identity_transform : 0;
  int64_t m = opts && opts->fit_sample > 0 ? std::min<int64_t>(opts->fit_sample, n)
                                           : std::min<int64_t>(n, 65536);
  std::vector<float> host;
  const float* Xh = X;
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, X) == cudaSuccess &&
      (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged)) {
    host.resize((size_t)m * d);
    PANO_CUDA(cudaMemcpy(host.data(), X, host.size() * 4, cudaMemcpyDeviceToHost));
    Xh = host.data();
  }
  cudaGetLastError();
  if (t->identity) {
    t->T.assign((size_t)d * d, 0.0);
    for (int i = 0; i < d; ++i) t->T[(size_t)i * d + i] = 1.0;
    t->mu.assign(d, 0.0);
    t->lam.assign(d, 0.0);
  } else {
    std::string err;
    int rc = fit_pca(Xh, m, d, t->mu, t->T, t->lam, err);
    if (rc) return fail(rc, err);
  }
  t->T32.resize((size_t)d * d);
  t->mu32.resize(d);
  for (size_t i = 0; i < t->T.size(); ++i) t->T32[i] = (float)t->T[i];
  for (int i = 0; i < d; ++i) t->mu32[i] = (float)t->mu[i];
  t->eta = t->identity ? 0.0 : orthogonality_defect(t->T32.data(), d) * (1.0 + 1e-6) + 1e-15;
  *out = t.release();
  return PANO_OK;
}

int panorama_transform_export(const pano_transform* t, double* T, double* mu, double* ev) {
  clear_error();
  PANO_CHECK(t, PANO_EINVAL, "null transform");
  if (T) std::memcpy(T, t->T.data(), t->T.size() * 8);
  if (mu) std::memcpy(mu, t->mu.data(), t->mu.size() * 8);
  if (ev) std::memcpy(ev, t->lam.data(), t->lam.size() * 8);
  return PANO_OK;
}

int panorama_transform_dim(const pano_transform* t) { return t ? t->d : 0; }
void panorama_free_transform(pano_transform* t) { delete t; }

int panorama_build_ivf(const pano_transform* t, const float* X, int64_t n, int32_t nlist,
                       const pano_build_opts* opts, void* stream, pano_index** out) {
  clear_error();
  return build_ivf(t, X, n, nlist, opts, (cudaStream_t)stream, out);
}

int panorama_search(const pano_index* idx, const float* queries, int64_t nq,
                    const int32_t* nprobe, int32_t nprobe_scalar, const int32_t* k,
                    int32_t k_scalar, int32_t k_max, int64_t* out_ids, float* out_dists,
                    void* stream) {
  clear_error();
  return search(idx, queries, nq, nprobe, nprobe_scalar, k, k_scalar, k_max, out_ids, out_dists,
                (cudaStream_t)stream, nullptr);
}

int panorama_search_ex(const pano_index* idx, const float* queries, int64_t nq,
                       const int32_t* nprobe, int32_t nprobe_scalar, const int32_t* k,
                       int32_t k_scalar, int32_t k_max, int64_t* out_ids, float* out_dists,
                       void* stream, const pano_search_opts* opts) {
  clear_error();
  return search(idx, queries, nq, nprobe, nprobe_scalar, k, k_scalar, k_max, out_ids, out_dists,
                (cudaStream_t)stream, opts);
}

int panorama_build_flat(const pano_transform* t, const float* X, int64_t n,
                        const pano_build_opts* opts, void* stream, pano_index** out) {
  clear_error();
  return build_flat(t, X, n, opts, (cudaStream_t)stream, out);
}

int panorama_refine(const pano_index* idx, const float* queries, int64_t nq,
                    const int64_t* cand_ids, int32_t kprime, int32_t k, int64_t* out_ids,
                    float* out_dists, float epsilon, void* stream) {
  clear_error();
  return refine(idx, queries, nq, cand_ids, kprime, k, out_ids, out_dists, epsilon,
                (cudaStream_t)stream);
}

int panorama_search_stats(pano_search_stats* out) {
  PANO_CHECK(out, PANO_EINVAL, "null stats");
  *out = last_stats();
  return PANO_OK;
}

int panorama_status_of_device_error(int32_t word) { return status_of_device_error(word); }

int panorama_probe(const pano_index* idx, const float* queries, int64_t nq, int32_t nprobe,
                   int32_t* out_lists, void* stream) {
  clear_error();
  return probe_only(idx, queries, nq, nprobe, out_lists, (cudaStream_t)stream);
}

int panorama_index_info(const pano_index* idx, pano_index_info* out) {
  clear_error();
  PANO_CHECK(idx && out, PANO_EINVAL, "null argument");
  out->n = idx->n;
  out->d = idx->d;
  out->nlist = idx->nlist;
  out->n_levels = idx->L;
  out->precision = idx->precision;
  out->chunk = idx->chunk;
  out->max_level_width = idx->max_w;
  out->n_chunks = idx->n_chunks;
  out->device_bytes = (int64_t)idx->device_bytes();
  out->eta = idx->eta;
  return PANO_OK;
}

int panorama_index_centroids(const pano_index* idx, float* out) {
  clear_error();
  PANO_CHECK(idx && out, PANO_EINVAL, "null argument");
  std::memcpy(out, idx->centroids.data(), idx->centroids.size() * 4);
  return PANO_OK;
}

int panorama_index_assignment(const pano_index* idx, int32_t* out) {
  clear_error();
  PANO_CHECK(idx && out, PANO_EINVAL, "null argument");
  std::memcpy(out, idx->assign.data(), idx->assign.size() * 4);
  return PANO_OK;
}

int panorama_save(const pano_index* idx, const char* path) {
  clear_error();
  PANO_CHECK(idx && path, PANO_EINVAL, "null argument");
  Writer w;
  w.f.open(path, std::ios::binary | std::ios::trunc);
  PANO_CHECK((bool)w.f, PANO_EINVAL, std::string("cannot open ") + path);
  w.f.write(kMagic, 8);
  uint32_t ver = kVersion;
  w.f.write(reinterpret_cast<const char*>(&ver), 4);
  const pano_index& I = *idx;
  w.pod(I.n);
  w.pod(I.d);
  w.pod(I.nlist);
  w.pod(I.L);
  w.pod(I.precision);
  w.pod(I.chunk);
  w.pod(I.max_w);
  w.pod(I.n_chunks);
  w.pod(I.eta);
  w.pod(I.c_trans);
  w.pod(I.cmax);
  w.vec(I.widths);
  w.vec(I.offs);
  w.pod(I.tf.d);
  w.pod(I.tf.identity);
  w.pod(I.tf.eta);
  w.vec(I.tf.T);
  w.vec(I.tf.mu);
  w.vec(I.tf.lam);
  w.vec(I.tf.T32);
  w.vec(I.tf.mu32);
  w.vec(I.centroids);
  w.vec(I.assign);
  w.vec(I.list_chunk_off);
  w.vec(I.list_size);
  int rc;
  if (I.precision == PANO_PQ) {  // the quantiser in place of the slices
    w.pod(I.pq_M);
    w.pod(I.pq_dsub);
    if ((rc = w.dev(I.pq_codes)) || (rc = w.dev(I.tails)) || (rc = w.dev(I.ids)) ||
        (rc = w.dev(I.pq_codebook)) || (rc = w.dev(I.pq_cent_t)))
      return rc;
  } else if ((rc = w.dev(I.slices)) || (rc = w.dev(I.tails)) || (rc = w.dev(I.xn2)) ||
             (rc = w.dev(I.ex)) || (rc = w.dev(I.ids)) || (rc = w.dev(I.rows)) ||
             (I.precision == PANO_FP8 && (rc = w.dev(I.xscale)))) {
    return rc;
  }
  uint64_t h = w.fnv.h;
  w.f.write(reinterpret_cast<const char*>(&h), 8);
  PANO_CHECK(w.ok && (bool)w.f, PANO_EINVAL, std::string("write failed: ") + path);
  return PANO_OK;
}

int panorama_load(const char* path, pano_index** out) {
  clear_error();
  PANO_CHECK(path && out, PANO_EINVAL, "null argument");
  int dev = 0;
  int rc = check_device(&dev);
  if (rc) return rc;
  Reader r;
  r.f.open(path, std::ios::binary | std::ios::ate);
  PANO_CHECK((bool)r.f, PANO_EINVAL, std::string("cannot open ") + path);
  uint64_t size = (uint64_t)r.f.tellg();
  r.f.seekg(0);
  PANO_CHECK(size >= 20, PANO_ECORRUPT, "file too short");
  char magic[8];
  uint32_t ver = 0;
  r.f.read(magic, 8);
  r.f.read(reinterpret_cast<char*>(&ver), 4);
  PANO_CHECK(std::memcmp(magic, kMagic, 8) == 0, PANO_ECORRUPT, "bad magic");
  PANO_CHECK(ver == kVersion, PANO_ECORRUPT, "unsupported version");
  r.remaining = size - 12 - 8;
  auto idx = std::make_unique<pano_index>();
  pano_index& I = *idx;
  I.device = dev;
  r.pod(I.n);
  r.pod(I.d);
  r.pod(I.nlist);
  r.pod(I.L);
  r.pod(I.precision);
  r.pod(I.chunk);
  r.pod(I.max_w);
  r.pod(I.n_chunks);
  r.pod(I.eta);
  r.pod(I.c_trans);
  r.pod(I.cmax);
  const bool sane = r.ok && I.n >= 1 && I.d >= 1 && I.d <= 65536 && I.nlist >= 1 &&
                    I.nlist <= I.n && I.L >= 1 && I.L <= 64 &&
                    ((I.precision == PANO_FP32 && I.chunk == 64) ||
                     ((I.precision == PANO_BF16 || I.precision == PANO_FP8) &&
                      I.chunk == 128) ||
                     (I.precision == PANO_FP32 && I.chunk == 1 && I.nlist == 1) ||
                     (I.precision == PANO_PQ && I.chunk == 256)) &&
                    I.n_chunks >= 0 && I.n_chunks <= I.n + I.nlist;
  PANO_CHECK(sane, PANO_ECORRUPT, "header fields out of range");
  I.flat = I.chunk == 1 ? 1 : 0;  // a flat (refine) index: one row per "chunk"
  const uint64_t d = I.d, n = I.n, nl = I.nlist;
  r.vec(I.widths, 64);
  r.vec(I.offs, 65);
  r.pod(I.tf.d);
  r.pod(I.tf.identity);
  r.pod(I.tf.eta);
  r.vec(I.tf.T, d * d);
  r.vec(I.tf.mu, d);
  r.vec(I.tf.lam, d);
  r.vec(I.tf.T32, d * d);
  r.vec(I.tf.mu32, d);
  r.vec(I.centroids, nl * d);
  r.vec(I.assign, n);
  r.vec(I.list_chunk_off, nl + 1);
  r.vec(I.list_size, nl);
  PANO_CHECK(r.ok && I.widths.size() == (size_t)I.L && I.offs.size() == (size_t)I.L + 1 &&
                 I.tf.T32.size() == d * d && I.centroids.size() == nl * d &&
                 I.assign.size() == n && I.list_chunk_off.size() == nl + 1 &&
                 I.list_chunk_off[nl] == I.n_chunks,
             PANO_ECORRUPT, "truncated or inconsistent index file");
  const uint64_t CHK = (uint64_t)I.chunk, ns = (uint64_t)I.n_chunks * CHK;
  if (I.precision == PANO_PQ) {
    r.pod(I.pq_M);
    r.pod(I.pq_dsub);
    const int M = I.pq_M, ds = I.pq_dsub;
    PANO_CHECK(r.ok && M >= 1 && ds >= 1 && ds <= 32 && (uint64_t)M * ds == d && M % I.L == 0 &&
                   M / I.L <= 64 && d % I.L == 0,
               PANO_ECORRUPT, "IVFPQ fields out of range");
    if ((rc = r.dev(I.pq_codes, ns * M)) || (rc = r.dev(I.tails, ns * I.L * 4)) ||
        (rc = r.dev(I.ids, ns * 4)) || (rc = r.dev(I.pq_codebook, (uint64_t)M * 256 * ds * 4)) ||
        (rc = r.dev(I.pq_cent_t, nl * d * 4)))
      return rc;
  } else if ((rc = r.dev(I.slices, I.slices_bytes())) ||
      (rc = r.dev(I.tails, (uint64_t)I.n_chunks * (I.L + 1) * CHK * 4)) ||
      (rc = r.dev(I.xn2, ns * 4)) || (rc = r.dev(I.ex, ns * 4)) || (rc = r.dev(I.ids, ns * 4)) ||
      (rc = r.dev(I.rows, ns * d * 4)) ||
      (I.precision == PANO_FP8 && (rc = r.dev(I.xscale, ns * 4))))
    return rc;
  PANO_CHECK(r.ok && r.remaining == 0, PANO_ECORRUPT, "truncated index file");
  uint64_t h = 0;
  r.f.read(reinterpret_cast<char*>(&h), 8);
  PANO_CHECK((bool)r.f && h == r.fnv.h, PANO_ECORRUPT, "checksum mismatch");
  // device copies of the small tables
  std::vector<float> hcn(I.nlist);
  for (int c = 0; c < I.nlist; ++c) {
    double s = 0;
    for (uint64_t j = 0; j < d; ++j) s += (double)I.centroids[c * d + j] * I.centroids[c * d + j];
    hcn[c] = (float)s;
  }
  if ((rc = I.cent.alloc(nl * d * 4)) || (rc = I.cent_n2.alloc(nl * 4)) ||
      (rc = I.chunk_off_d.alloc((nl + 1) * 8)) || (rc = I.list_size_d.alloc(nl * 4)) ||
      (rc = I.level_off_d.alloc((I.L + 1) * 4)) || (rc = I.T32.alloc(d * d * 4)) ||
      (rc = I.mu32.alloc(d * 4)))
    return rc;
  PANO_CUDA(cudaMemcpy(I.cent.p, I.centroids.data(), nl * d * 4, cudaMemcpyHostToDevice));
  PANO_CUDA(cudaMemcpy(I.cent_n2.p, hcn.data(), nl * 4, cudaMemcpyHostToDevice));
  PANO_CUDA(cudaMemcpy(I.chunk_off_d.p, I.list_chunk_off.data(), (nl + 1) * 8, cudaMemcpyHostToDevice));
  PANO_CUDA(cudaMemcpy(I.list_size_d.p, I.list_size.data(), nl * 4, cudaMemcpyHostToDevice));
  PANO_CUDA(cudaMemcpy(I.level_off_d.p, I.offs.data(), (I.L + 1) * 4, cudaMemcpyHostToDevice));
  PANO_CUDA(cudaMemcpy(I.T32.p, I.tf.T32.data(), d * d * 4, cudaMemcpyHostToDevice));
  PANO_CUDA(cudaMemcpy(I.mu32.p, I.tf.mu32.data(), d * 4, cudaMemcpyHostToDevice));
  *out = idx.release();
  return PANO_OK;
}

void panorama_free_index(pano_index* idx) {
  if (!idx) return;
  int cur = 0;
  const int dev = idx->device;
  cudaGetDevice(&cur);
  if (cur != dev) cudaSetDevice(dev);
  delete idx;
  if (cur != dev) cudaSetDevice(cur);
}

}  // extern "C"
