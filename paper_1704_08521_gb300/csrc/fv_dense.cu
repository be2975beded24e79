// Small dense FP64 routines on the m x m (m <= 128) upper Hessenberg matrix
// of the Arnoldi factorisation (Section 3: Arnoldi in regular mode, ARPACK /
// Sorensen 1992 implicit restarts):
//   * eigenvalues by the Francis double-shift QR iteration with deflation
//     (Golub & Van Loan, Algorithms 7.5.1-7.5.2);
//   * one implicit double-shift step (a complex-conjugate pair of shifts) or
//     one single-shift Givens bulge chase (a real shift), accumulating Q;
//   * an eigenvector of H for a given eigenvalue by complex inverse iteration.
#include <cmath>
#include <complex>
#include <vector>

#include "fv_ff.cuh"
#include "fv_internal.cuh"

namespace fv {

namespace {

// Householder vector v (v[0] = 1) and beta with (I - beta v v^T) x = +-||x|| e1.
void house(int len, const double* x, double* v, double& beta) {
  double sigma = 0.0;
  for (int i = 1; i < len; ++i) sigma += x[i] * x[i];
  v[0] = 1.0;
  for (int i = 1; i < len; ++i) v[i] = x[i];
  if (sigma == 0.0) { beta = 0.0; return; }
  const double mu = std::sqrt(x[0] * x[0] + sigma);
  const double v0 = (x[0] <= 0.0) ? x[0] - mu : -sigma / (x[0] + mu);
  beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
  for (int i = 1; i < len; ++i) v[i] = x[i] / v0;
}

// Apply P = I - beta v v^T (len 2 or 3, acting on indices k..k+len-1) as a
// similarity to H (rows from column c0, columns up to row r1) and to Q.
void apply_reflector(int m, double* H, double* Q, int k, int len, const double* v, double beta,
                     int c0, int r1) {
  if (beta == 0.0) return;
  for (int c = c0; c < m; ++c) {
    double s = 0.0;
    for (int i = 0; i < len; ++i) s += v[i] * H[(k + i) * m + c];
    s *= beta;
    for (int i = 0; i < len; ++i) H[(k + i) * m + c] -= s * v[i];
  }
  for (int r = 0; r <= r1; ++r) {
    double s = 0.0;
    for (int i = 0; i < len; ++i) s += H[r * m + k + i] * v[i];
    s *= beta;
    for (int i = 0; i < len; ++i) H[r * m + k + i] -= s * v[i];
  }
  if (Q) {
    for (int r = 0; r < m; ++r) {
      double s = 0.0;
      for (int i = 0; i < len; ++i) s += Q[r * m + k + i] * v[i];
      s *= beta;
      for (int i = 0; i < len; ++i) Q[r * m + k + i] -= s * v[i];
    }
  }
}

// Francis double-shift step on the unreduced block lo..hi (hi - lo >= 2)
// for the shift pair mid +- sqrt(disc) (disc < 0: a complex pair).  The
// first column of (H - r1)(H - r2) is formed from the differences
// h_ii - mid: expanding it through the sum and product of the shifts loses
// everything when the block is close to a multiple of the identity.
void francis_block(int m, double* H, double* Q, int lo, int hi, double mid, double disc) {
  auto a = [&](int i, int j) { return H[i * m + j]; };
  const double d0 = a(lo, lo) - mid, d1 = a(lo + 1, lo + 1) - mid;
  double x = d0 * d0 - disc + a(lo, lo + 1) * a(lo + 1, lo);
  double y = a(lo + 1, lo) * (d0 + d1);
  double z = a(lo + 1, lo) * a(lo + 2, lo + 1);
  double v[3], beta;
  for (int k = lo; k <= hi - 2; ++k) {
    const double xv[3] = {x, y, z};
    house(3, xv, v, beta);
    const int c0 = (k - 1 > lo) ? k - 1 : lo;
    const int r1 = (k + 3 < hi) ? k + 3 : hi;
    apply_reflector(m, H, Q, k, 3, v, beta, c0, r1);
    x = a(k + 1, k);
    y = a(k + 2, k);
    if (k < hi - 2) z = a(k + 3, k);
  }
  const double xv[2] = {x, y};
  house(2, xv, v, beta);
  apply_reflector(m, H, Q, hi - 1, 2, v, beta, hi - 2, hi);
  // the bulge chase leaves exact zeros below the subdiagonal up to round-off
  for (int i = lo + 2; i <= hi; ++i)
    for (int j = lo; j < i - 1; ++j) H[i * m + j] = 0.0;
}

}  // namespace

bool hess_eigenvalues(int m, const double* H0, double* wr, double* wi) {
  std::vector<double> A(H0, H0 + (size_t)m * m);
  double* H = A.data();
  auto a = [&](int i, int j) -> double& { return H[i * m + j]; };
  double hnorm = 0.0;
  for (int i = 0; i < m * m; ++i) hnorm = std::fmax(hnorm, std::fabs(A[i]));
  const double eps = 2.2204460492503131e-16;
  int hi = m - 1, its = 0, total = 0;
  while (hi >= 0) {
    int lo = hi;
    while (lo > 0) {
      double sc = std::fabs(a(lo - 1, lo - 1)) + std::fabs(a(lo, lo));
      if (sc == 0.0) sc = hnorm;
      if (std::fabs(a(lo, lo - 1)) <= eps * sc) { a(lo, lo - 1) = 0.0; break; }
      --lo;
    }
    if (lo == hi) {
      wr[hi] = a(hi, hi); wi[hi] = 0.0;
      --hi; its = 0;
      continue;
    }
    if (lo == hi - 1) {
      const double p = a(hi - 1, hi - 1), q = a(hi - 1, hi), r = a(hi, hi - 1), s = a(hi, hi);
      const double mid = 0.5 * (p + s);
      const double disc = 0.25 * (p - s) * (p - s) + q * r;
      if (disc >= 0.0) {
        const double sq = std::sqrt(disc);
        const double l1 = mid + (mid >= 0 ? sq : -sq);
        const double l2 = (l1 != 0.0) ? (p * s - q * r) / l1 : mid - sq;
        wr[hi - 1] = l1; wi[hi - 1] = 0.0;
        wr[hi] = l2; wi[hi] = 0.0;
      } else {
        const double im = std::sqrt(-disc);
        wr[hi - 1] = mid; wi[hi - 1] = im;
        wr[hi] = mid; wi[hi] = -im;
      }
      hi -= 2; its = 0;
      continue;
    }
    if (++total > 60 * m) return false;
    ++its;
    double mid, disc;
    if (its % 11 == 10) {
      // exceptional shift pair a_hh + 0.75 x +- 0.66 i x, x the size of the
      // last two subdiagonal entries, to break a cycle of the standard shifts
      const double x = std::fabs(a(hi, hi - 1)) + std::fabs(a(hi - 1, hi - 2));
      mid = a(hi, hi) + 0.75 * x;
      disc = -0.4375 * x * x;
    } else {
      // the eigenvalues of the trailing 2 x 2 block
      const double hd = 0.5 * (a(hi - 1, hi - 1) - a(hi, hi));
      mid = 0.5 * (a(hi - 1, hi - 1) + a(hi, hi));
      disc = hd * hd + a(hi - 1, hi) * a(hi, hi - 1);
    }
    francis_block(m, H, nullptr, lo, hi, mid, disc);
  }
  return true;
}

void francis_double_step(int m, double* H, double* Q, double re, double im) {
  if (m < 3) return;
  francis_block(m, H, Q, 0, m - 1, re, -im * im);
}

void single_shift_step(int m, double* H, double* Q, double mu) {
  double x = H[0] - mu, y = H[m];
  for (int k = 0; k < m - 1; ++k) {
    const double r = std::hypot(x, y);
    double c = 1.0, s = 0.0;
    if (r != 0.0) { c = x / r; s = y / r; }
    const int c0 = (k - 1 > 0) ? k - 1 : 0;
    for (int j = c0; j < m; ++j) {            // rows k, k+1  (G^T from the left)
      const double t0 = H[k * m + j], t1 = H[(k + 1) * m + j];
      H[k * m + j] = c * t0 + s * t1;
      H[(k + 1) * m + j] = -s * t0 + c * t1;
    }
    const int r1 = (k + 2 < m - 1) ? k + 2 : m - 1;
    for (int i = 0; i <= r1; ++i) {           // columns k, k+1
      const double t0 = H[i * m + k], t1 = H[i * m + k + 1];
      H[i * m + k] = c * t0 + s * t1;
      H[i * m + k + 1] = -s * t0 + c * t1;
    }
    for (int i = 0; i < m; ++i) {
      const double t0 = Q[i * m + k], t1 = Q[i * m + k + 1];
      Q[i * m + k] = c * t0 + s * t1;
      Q[i * m + k + 1] = -s * t0 + c * t1;
    }
    if (k < m - 2) { x = H[(k + 1) * m + k]; y = H[(k + 2) * m + k]; }
  }
  for (int i = 2; i < m; ++i)
    for (int j = 0; j < i - 1; ++j) H[i * m + j] = 0.0;
}

void hess_eigvec(int m, const double* H, double tr, double ti, double* yr, double* yi) {
  using cd = std::complex<double>;
  std::vector<cd> A((size_t)m * m);
  double hnorm = 0.0;
  for (int i = 0; i < m * m; ++i) hnorm = std::fmax(hnorm, std::fabs(H[i]));
  const cd theta(tr, ti);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[i * m + j] = cd(H[i * m + j]) - (i == j ? theta : cd(0.0));
  // LU with partial pivoting
  std::vector<int> piv(m);
  const double tiny = 1e-14 * (hnorm > 0 ? hnorm : 1.0);
  for (int k = 0; k < m; ++k) {
    int p = k;
    for (int i = k + 1; i < m; ++i)
      if (std::abs(A[i * m + k]) > std::abs(A[p * m + k])) p = i;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < m; ++j) std::swap(A[k * m + j], A[p * m + j]);
    if (std::abs(A[k * m + k]) < tiny) A[k * m + k] = tiny;
    for (int i = k + 1; i < m; ++i) {
      const cd f = A[i * m + k] / A[k * m + k];
      A[i * m + k] = f;
      for (int j = k + 1; j < m; ++j) A[i * m + j] -= f * A[k * m + j];
    }
  }
  std::vector<cd> y(m, cd(1.0, 0.0));
  for (int it = 0; it < 3; ++it) {
    for (int k = 0; k < m; ++k)
      if (piv[k] != k) std::swap(y[k], y[piv[k]]);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < i; ++j) y[i] -= A[i * m + j] * y[j];
    for (int i = m - 1; i >= 0; --i) {
      for (int j = i + 1; j < m; ++j) y[i] -= A[i * m + j] * y[j];
      y[i] /= A[i * m + i];
    }
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += std::norm(y[i]);
    nrm = std::sqrt(nrm);
    for (int i = 0; i < m; ++i) y[i] /= nrm;
  }
  for (int i = 0; i < m; ++i) { yr[i] = y[i].real(); yi[i] = y[i].imag(); }
}

}  // namespace fv

// ---- host-only entry points used by the CPU tests of this logic ----------
extern "C" int fv_host_hess_eigenvalues(int m, const double* H, double* wr, double* wi) {
  if (m < 1 || m > 512 || !H || !wr || !wi) return FV_EINVAL;
  return fv::hess_eigenvalues(m, H, wr, wi) ? FV_OK : FV_ENOCONV;
}

extern "C" int fv_host_shift_steps(int m, double* H, double* Q, int nshift, const double* sr,
                                   const double* si) {
  if (m < 3 || m > 512 || !H || !Q) return FV_EINVAL;
  for (int i = 0; i < nshift; ++i) {
    if (si[i] != 0.0 && i + 1 < nshift && si[i + 1] == -si[i] && sr[i + 1] == sr[i]) {
      fv::francis_double_step(m, H, Q, sr[i], si[i]);
      ++i;
    } else {
      fv::single_shift_step(m, H, Q, sr[i]);
    }
  }
  return FV_OK;
}

// Float-float conversions of the mixed-precision path, host build of the
// same integer routines the kernels use (for CPU tests).
extern "C" int fv_host_ff_convert(int64_t n, const double* in, float* hi, float* lo,
                                  double* joined, float* rounded) {
  if (n < 0 || !in) return FV_EINVAL;
  for (int64_t i = 0; i < n; ++i) {
    const fv::ff s = fv::f64_split(in[i]);
    if (hi) hi[i] = s.hi;
    if (lo) lo[i] = s.lo;
    if (joined) joined[i] = fv::ff_join(s.hi, s.lo);
    if (rounded) rounded[i] = fv::f64_round_f32(in[i]);
  }
  return FV_OK;
}

// the Krylov-basis kernels' float-float dot product on the host:
// out = sum_i a_i b_i with the truncating split and the multiply-add
extern "C" int fv_host_ff_dot(int64_t n, const double* a, const double* b, double* out) {
  if (n < 0 || !a || !b || !out) return FV_EINVAL;
  fv::ff acc{0.0f, 0.0f};
  for (int64_t i = 0; i < n; ++i) fv::ff_mad(acc, fv::f64_split_trunc(a[i]), fv::f64_split_trunc(b[i]));
  *out = fv::ff_join(acc.hi, acc.lo);
  return FV_OK;
}

// ff arithmetic on the host: out = (a + b) * c with a, b, c given as (hi, lo)
extern "C" int fv_host_ff_arith(int64_t n, const float* a, const float* b, const float* c,
                                float* out) {
  for (int64_t i = 0; i < n; ++i) {
    const fv::ff x{a[2 * i], a[2 * i + 1]}, y{b[2 * i], b[2 * i + 1]}, z{c[2 * i], c[2 * i + 1]};
    const fv::ff r = fv::ff_mul(fv::ff_add(x, y), z);
    out[2 * i] = r.hi;
    out[2 * i + 1] = r.lo;
  }
  return FV_OK;
}
