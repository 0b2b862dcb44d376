// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/panorama.h"

namespace pano {

// ------------------------------------------------------------ error state
void set_error(const std::string& msg);
void clear_error();
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define PANO_CUDA(expr)                                   \
  do {                                                    \
    cudaError_t e_ = (expr);                              \
    if (e_ != cudaSuccess) return ::pano::cuda_fail(e_, #expr); \
  } while (0)

#define PANO_CHECK(cond, code, msg)          \
  do {                                       \
    if (!(cond)) return ::pano::fail(code, msg); \
  } while (0)

// ------------------------------------------------ rounding-error constants
// Unit roundoff of FP32 (round to nearest).
constexpr double kU32 = 5.9604644775390625e-08;  // 2^-24
// gamma_n = n u / (1 - n u): bound on the relative error of an n-term
// floating-point sum/product chain (standard a priori analysis).
inline double gamma_n(double n) { return n * kU32 / (1.0 - n * kU32); }

// The SIMT GEMM accumulates each K-tile of GEMM_KT products in a fresh
// register and then adds the tile sums, so every product passes through at
// most GEMM_KT + ceil(K / GEMM_KT) + 1 roundings.
constexpr int GEMM_KT = 16;
inline double gemm_rounds(int K) { return GEMM_KT + (K + GEMM_KT - 1) / GEMM_KT + 1; }

// ------------------------------------------------------------ host helpers
// Runs a set-up step once per device (the current one at the call): kernel
// attributes such as the dynamic shared-memory limit belong to the device's
// context, so a process that searches on several devices sets them on each.
// Returns that device's result (an error is kept, not retried).
class PerDeviceOnce {
 public:
  template <class F>
  cudaError_t run(F&& setup) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu_);
    if (!done_[dev]) {
      err_[dev] = setup();
      done_[dev] = true;
    }
    return err_[dev];
  }

 private:
  static constexpr int kMaxDevices = 64;
  std::mutex mu_;
  bool done_[kMaxDevices] = {};
  cudaError_t err_[kMaxDevices] = {};
};

void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& fn);
int fit_pca(const float* X, int64_t n, int d, std::vector<double>& mu,
            std::vector<double>& T, std::vector<double>& lam, std::string& err);
double orthogonality_defect(const float* A, int d);

// Device allocation owned by an index (freed in the destructor).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  int alloc(size_t n);
  void release();
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
  ~DevBuf() { release(); }
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

}  // namespace pano

struct pano_transform {
  int32_t d = 0;
  int32_t identity = 0;
  std::vector<double> T, mu, lam;  // FP64 fit
  std::vector<float> T32, mu32;    // what the device uses (T~, mu~)
  double eta = 0.0;                // ||T~^T T~ - I||_F (bounds sigma(T~))
};

struct pano_index {
  int device = 0;
  int64_t n = 0;
  int32_t d = 0, nlist = 0, L = 0, precision = 0, chunk = 64;
  int32_t max_w = 0;
  // 1: flat row-major index for refining candidate-id lists (B = 1): slices
  // holds the x~ rows [n][d] FP32, tails [n][L+1], xn2 / ex [n], rows [n][d]
  // the original rows; the id of a vector is its row.  0: IVF, level-major.
  int32_t flat = 0;
  std::vector<int32_t> widths, offs;  // offs[l] = m_l, l = 0..L
  int64_t n_chunks = 0;
  double eta = 0.0;     // orthogonality defect of T~
  double c_trans = 0.0; // e(v) <= c_trans * ||v - mu~|| for the FP32 transform
  float cmax = 0.f;     // max centroid norm (probe rounding band)
  pano_transform tf;
  // host copies
  std::vector<float> centroids;         // nlist x d, original space
  std::vector<int32_t> assign;          // n: list of each vector
  std::vector<int64_t> list_chunk_off;  // nlist + 1
  std::vector<int32_t> list_size;       // nlist
  // device arrays
  pano::DevBuf T32, mu32;        // d x d, d
  pano::DevBuf cent, cent_n2;    // nlist x d, nlist   (original space)
  pano::DevBuf chunk_off_d;      // nlist + 1 int64
  pano::DevBuf list_size_d;      // nlist int32
  pano::DevBuf level_off_d;      // L + 1 int32 (m_l)
  // FP32: per chunk, per level l a block of [w_l + 1][64] floats (the level
  // slice, dims-major, then the tail column sqrt(R^{(l+1,d)})); level 0's
  // block has three more rows (||x~||^2, e_x, id bits).  BF16 / FP8: see
  // verify_tc.
  pano::DevBuf slices;
  pano::DevBuf tails;    // [chunk][L+1][CH] sqrt tail energy, rounded up
  pano::DevBuf xn2;      // [chunk][CH] ||x~||^2
  pano::DevBuf ex;       // [chunk][CH] bound on ||x~ - T~(x - mu~)||
  pano::DevBuf ids;      // [chunk][CH] int32 original id, -1 = padding
  pano::DevBuf xscale;   // FP8: [chunk][CH] power-of-two scale s_x of each vector
  pano::DevBuf rows;     // [chunk * CH][d] original FP32 rows (re-ranking)
  // IVFPQ (precision PANO_PQ, chunk = 256): codes [block][M][256] u8, tails
  // [block][L][256] (in `tails`), ids [block][256] (in `ids`), the codebooks
  // [M][256][dsub] and the transformed centroids [nlist][d]
  int32_t pq_M = 0, pq_dsub = 0;
  pano::DevBuf pq_codes, pq_codebook, pq_cent_t;
  size_t device_bytes() const;
  // FP32 slice layout: rows (of 64 floats) per chunk, and the first row of
  // level l's block within a chunk
  int64_t fp32_chunk_rows() const { return (int64_t)d + L + 3; }
  int32_t fp32_row_off(int l) const { return l == 0 ? 0 : offs[l] + l + 3; }
  size_t slices_bytes() const {
    if (flat) return (size_t)n * d * 4;
    if (pq_M) return 0;
    return precision == PANO_FP32  ? (size_t)n_chunks * chunk * fp32_chunk_rows() * 4
           : precision == PANO_BF16 ? (size_t)n_chunks * chunk * d * 2
                                    : (size_t)n_chunks * chunk * d;
  }
};
