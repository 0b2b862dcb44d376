// Host-side FP64 PCA fit (Section 4.1 of the paper: the rows of T are the
// eigenvectors of the empirical covariance, ordered by eigenvalue
// descending).
//
// Steps: FP64 mean and covariance (1/n normalisation) -> Householder
// reduction to tridiagonal form with the reflections accumulated -> implicit
// QL iterations with a Wilkinson-type shift on the tridiagonal matrix, whose
// plane rotations are recorded and then applied to the accumulated basis in
// parallel over row blocks (rotations act on columns, so rows are
// independent).  Both are the textbook dense symmetric eigen-solver.
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

namespace pano {

void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& fn) {
  int64_t nt = std::max(1u, std::thread::hardware_concurrency());
  nt = std::min<int64_t>(nt, 64);
  if (n < 2 || nt == 1) {
    fn(0, n);
    return;
  }
  nt = std::min(nt, n);
  std::vector<std::thread> th;
  int64_t per = (n + nt - 1) / nt;
  for (int64_t t = 0; t < nt; ++t) {
    int64_t b = t * per, e = std::min(n, b + per);
    if (b >= e) break;
    th.emplace_back([=, &fn] { fn(b, e); });
  }
  for (auto& x : th) x.join();
}

// Covariance of the rows of X (n x d FP32) about their FP64 mean.
static void covariance(const float* X, int64_t n, int d, std::vector<double>& mu,
                       std::vector<double>& C) {
  mu.assign(d, 0.0);
  int nt = std::max(1u, std::thread::hardware_concurrency());
  nt = std::min(nt, 64);
  std::vector<std::vector<double>> part_mu(nt, std::vector<double>(d, 0.0));
  int64_t per = (n + nt - 1) / nt;
  parallel_for(nt, [&](int64_t b, int64_t e) {
    for (int64_t t = b; t < e; ++t) {
      int64_t r0 = t * per, r1 = std::min(n, r0 + per);
      double* m = part_mu[t].data();
      for (int64_t r = r0; r < r1; ++r)
        for (int j = 0; j < d; ++j) m[j] += X[r * (int64_t)d + j];
    }
  });
  for (int t = 0; t < nt; ++t)
    for (int j = 0; j < d; ++j) mu[j] += part_mu[t][j];
  for (int j = 0; j < d; ++j) mu[j] /= (double)n;

  // each thread accumulates the upper triangle of its rows' outer products
  std::vector<std::vector<double>> part(nt);
  parallel_for(nt, [&](int64_t b, int64_t e) {
    for (int64_t t = b; t < e; ++t) {
      std::vector<double>& P = part[t];
      P.assign((size_t)d * d, 0.0);
      int64_t r0 = t * per, r1 = std::min(n, r0 + per);
      std::vector<double> xc(4 * (size_t)d);
      int64_t r = r0;
      for (; r + 4 <= r1; r += 4) {  // four rows at a time
        for (int q = 0; q < 4; ++q)
          for (int j = 0; j < d; ++j)
            xc[q * d + j] = (double)X[(r + q) * (int64_t)d + j] - mu[j];
        for (int a = 0; a < d; ++a) {
          double x0 = xc[a], x1 = xc[d + a], x2 = xc[2 * d + a],
                 x3 = xc[3 * d + a];
          double* row = P.data() + (size_t)a * d;
          for (int c = a; c < d; ++c)
            row[c] += x0 * xc[c] + x1 * xc[d + c] + x2 * xc[2 * d + c] +
                      x3 * xc[3 * d + c];
        }
      }
      for (; r < r1; ++r) {
        for (int j = 0; j < d; ++j)
          xc[j] = (double)X[r * (int64_t)d + j] - mu[j];
        for (int a = 0; a < d; ++a) {
          double* row = P.data() + (size_t)a * d;
          for (int c = a; c < d; ++c) row[c] += xc[a] * xc[c];
        }
      }
    }
  });
  C.assign((size_t)d * d, 0.0);
  for (int t = 0; t < nt; ++t) {
    if (part[t].empty()) continue;
    for (size_t i = 0; i < C.size(); ++i) C[i] += part[t][i];
  }
  for (int a = 0; a < d; ++a)
    for (int c = a; c < d; ++c) {
      double v = C[(size_t)a * d + c] / (double)n;
      C[(size_t)a * d + c] = v;
      C[(size_t)c * d + a] = v;
    }
}

// Householder reduction of symmetric A (n x n, destroyed) to tridiagonal
// form: Q^T A Q = tridiag(diag, off).  Q (row-major n x n) accumulates the
// reflections.  off[i] couples i and i+1.
static void tridiagonalize(std::vector<double>& A, int n, std::vector<double>& diag,
                           std::vector<double>& off, std::vector<double>& Q) {
  diag.assign(n, 0.0);
  off.assign(n, 0.0);
  std::vector<std::vector<double>> vs(n);
  std::vector<double> beta(n, 0.0), p(n), w(n);
  for (int k = 0; k + 2 < n; ++k) {
    int m = n - k - 1;  // length of the sub-column below the diagonal
    std::vector<double>& v = vs[k];
    v.assign(m, 0.0);
    double norm2 = 0.0;
    for (int i = 0; i < m; ++i) {
      v[i] = A[(size_t)(k + 1 + i) * n + k];
      norm2 += v[i] * v[i];
    }
    double alpha = std::sqrt(norm2);
    if (alpha == 0.0) {
      beta[k] = 0.0;
      off[k] = 0.0;
      continue;
    }
    if (v[0] > 0) alpha = -alpha;  // reflect onto -sign(x0) ||x|| e1
    v[0] -= alpha;
    double vtv = 0.0;
    for (int i = 0; i < m; ++i) vtv += v[i] * v[i];
    if (vtv == 0.0) {
      beta[k] = 0.0;
      off[k] = alpha;
      continue;
    }
    double b = 2.0 / vtv;
    beta[k] = b;
    off[k] = alpha;
    // p = b * A_sub v ; K = b/2 * v^T p ; w = p - K v ; A_sub -= v w^T + w v^T
    const int o = k + 1;
    for (int i = 0; i < m; ++i) {
      const double* row = A.data() + (size_t)(o + i) * n + o;
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += row[j] * v[j];
      p[i] = b * s;
    }
    double vp = 0.0;
    for (int i = 0; i < m; ++i) vp += v[i] * p[i];
    double K = 0.5 * b * vp;
    for (int i = 0; i < m; ++i) w[i] = p[i] - K * v[i];
    for (int i = 0; i < m; ++i) {
      double* row = A.data() + (size_t)(o + i) * n + o;
      for (int j = 0; j < m; ++j) row[j] -= v[i] * w[j] + w[i] * v[j];
    }
  }
  for (int i = 0; i < n; ++i) diag[i] = A[(size_t)i * n + i];
  if (n >= 2) off[n - 2] = A[(size_t)(n - 1) * n + (n - 2)];
  off[n - 1] = 0.0;
  // Q = H_0 H_1 ... H_{n-3}, accumulated from the last reflection backwards
  Q.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  std::vector<double> t(n);
  for (int k = n - 3; k >= 0; --k) {
    if (beta[k] == 0.0) continue;
    const std::vector<double>& v = vs[k];
    int m = n - k - 1, o = k + 1;
    // Q_sub -= beta v (v^T Q_sub), Q_sub = Q[o:, o:]
    std::fill(t.begin(), t.begin() + m, 0.0);
    for (int i = 0; i < m; ++i) {
      const double* row = Q.data() + (size_t)(o + i) * n + o;
      double vi = v[i];
      for (int j = 0; j < m; ++j) t[j] += vi * row[j];
    }
    for (int i = 0; i < m; ++i) {
      double* row = Q.data() + (size_t)(o + i) * n + o;
      double s = beta[k] * v[i];
      for (int j = 0; j < m; ++j) row[j] -= s * t[j];
    }
  }
}

struct Rot {
  int32_t i;
  double c, s;
};

// Implicit QL with shifts on tridiag(diag, off); the plane rotations that
// act on columns (i, i+1) of the basis are appended to `rots`.
static bool tridiagonal_ql(std::vector<double>& dg, std::vector<double>& e, int n,
                           std::vector<Rot>& rots) {
  const double eps = std::numeric_limits<double>::epsilon();
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    while (true) {
      int m = l;
      for (; m < n - 1; ++m) {
        double dd = std::fabs(dg[m]) + std::fabs(dg[m + 1]);
        if (std::fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      if (++iter > 200) return false;
      // shift from the leading 2x2 block, closest eigenvalue to dg[l]
      double g = (dg[l + 1] - dg[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = dg[m] - dg[l] + e[l] / (g + std::copysign(r, g));
      double s = 1.0, c = 1.0, p = 0.0;
      bool deflated = false;
      for (int i = m - 1; i >= l; --i) {
        double f = s * e[i], b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {  // underflow: split the matrix and restart
          dg[i + 1] -= p;
          e[m] = 0.0;
          deflated = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = dg[i + 1] - p;
        r = (dg[i] - g) * s + 2.0 * c * b;
        p = s * r;
        dg[i + 1] = g + p;
        g = c * r - b;
        rots.push_back(Rot{i, c, s});
      }
      if (deflated) continue;
      dg[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  return true;
}

int fit_pca(const float* X, int64_t n, int d, std::vector<double>& mu,
            std::vector<double>& T, std::vector<double>& lam, std::string& err) {
  std::vector<double> C;
  covariance(X, n, d, mu, C);
  std::vector<double> diag, off, Q;
  tridiagonalize(C, d, diag, off, Q);
  std::vector<Rot> rots;
  rots.reserve((size_t)d * d * 2);
  if (!tridiagonal_ql(diag, off, d, rots)) {
    err = "eigen-solver did not converge";
    return PANO_EINVAL;
  }
  // apply the recorded rotations to Q's columns, rows in parallel
  parallel_for(d, [&](int64_t b, int64_t e) {
    for (int64_t r = b; r < e; ++r) {
      double* row = Q.data() + (size_t)r * d;
      for (const Rot& R : rots) {
        double f = row[R.i + 1];
        row[R.i + 1] = R.s * row[R.i] + R.c * f;
        row[R.i] = R.c * row[R.i] - R.s * f;
      }
    }
  });
  // columns of Q are eigenvectors; order by eigenvalue descending (stable)
  std::vector<int> order(d);
  for (int i = 0; i < d; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return diag[a] > diag[b]; });
  T.assign((size_t)d * d, 0.0);
  lam.assign(d, 0.0);
  for (int r = 0; r < d; ++r) {
    int c = order[r];
    lam[r] = diag[c];
    int arg = 0;
    double best = -1.0;
    for (int j = 0; j < d; ++j) {
      double v = std::fabs(Q[(size_t)j * d + c]);
      if (v > best) {
        best = v;
        arg = j;
      }
    }
    double sgn = Q[(size_t)arg * d + c] < 0 ? -1.0 : 1.0;
    for (int j = 0; j < d; ++j) T[(size_t)r * d + j] = sgn * Q[(size_t)j * d + c];
  }
  return PANO_OK;
}

// ||A^T A - I||_F for the FP32-rounded matrix A (d x d), in FP64.
double orthogonality_defect(const float* A, int d) {
  std::vector<double> At((size_t)d * d);  // columns of A as rows
  for (int k = 0; k < d; ++k)
    for (int i = 0; i < d; ++i) At[(size_t)i * d + k] = A[(size_t)k * d + i];
  std::vector<double> rowsum(d, 0.0);
  parallel_for(d, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      const double* ci = At.data() + (size_t)i * d;
      double acc = 0.0;
      for (int j = 0; j < d; ++j) {
        const double* cj = At.data() + (size_t)j * d;
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += ci[k] * cj[k];
        if (i == j) s -= 1.0;
        acc += s * s;
      }
      rowsum[i] = acc;
    }
  });
  double t = 0.0;
  for (double v : rowsum) t += v;
  return std::sqrt(t);
}

}  // namespace pano
