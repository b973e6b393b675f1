// Eigenvalues of the TSL tridiagonal T_k on the host (the Ritz values), for the
// run diagnostics: min |Re lambda(T_k)| tells how close the k x k sign problem
// is to ill-posed (sgn is undefined on the imaginary axis, Sec. 2 Eq.
// spectral_form).
//
// T_k has diagonal alpha_j, superdiagonal beta_{j+1} and subdiagonal delta_{j+1}
// with |beta_{j+1}| = |delta_{j+1}| (delta = sqrt|omega|, beta = omega / delta).
// A diagonal similarity with unimodular entries therefore turns it into the
// complex-symmetric tridiagonal S with off-diagonal e_j = sqrt(beta_{j+1} delta_{j+1})
// and the same eigenvalues, without any growth from the scaling.  S is reduced
// by the implicit QL iteration with a Wilkinson-type shift (Bowdler, Martin,
// Reinsch and Wilkinson, Numer. Math. 11 (1968) 293), run in complex arithmetic
// with complex-orthogonal plane rotations (c^2 + s^2 = 1), which keep S complex
// symmetric and tridiagonal (Cullum and Willoughby, "A QL procedure for
// computing the eigenvalues of complex symmetric tridiagonal matrices", SIAM J.
// Matrix Anal. Appl. 17 (1996) 83).  Each iteration costs O(k), the whole
// spectrum O(k^2).  Complex-orthogonal rotations are not unitary: a rotation
// whose normaliser sqrt(f^2 + g^2) nearly vanishes is reported as a failure
// instead of being taken.
#include <cmath>
#include <complex>
#include <vector>

#include "ov.h"

namespace {

using cx = std::complex<double>;

// sqrt(a^2 + b^2) for complex a, b, scaled against overflow; the branch is
// immaterial (it only flips the sign of a rotation)
cx hyp(cx a, cx b) {
  const double m = std::max(std::abs(a), std::abs(b));
  if (m == 0.0) return cx(0.0, 0.0);
  const cx x = a / m, y = b / m;
  return m * std::sqrt(x * x + y * y);
}

// Eigenvalues of the complex-symmetric tridiagonal (d, e) in place (d), e[n-1] unused.
// Returns false when the iteration does not converge or a rotation breaks down.
bool ql_complex_symmetric(std::vector<cx>& d, std::vector<cx>& e) {
  const int n = (int)d.size();
  const double eps = 2.220446049250313e-16;
  if (n <= 1) return true;
  e[n - 1] = 0.0;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    for (;;) {
      // the first negligible off-diagonal entry at or after l splits the matrix
      int m = l;
      for (; m < n - 1; ++m) {
        const double dd = std::abs(d[m]) + std::abs(d[m + 1]);
        if (std::abs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      if (++iter > 60) return false;
      // shift: the eigenvalue of the leading 2 x 2 block [[d_l, e_l], [e_l, d_{l+1}]]
      // nearer to d_l, expressed through g = (d_{l+1} - d_l) / (2 e_l)
      cx g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      cx r = hyp(g, cx(1.0, 0.0));
      const cx gp = (std::abs(g + r) >= std::abs(g - r)) ? g + r : g - r;
      g = d[m] - d[l] + e[l] / gp;
      if (iter == 20 || iter == 40) g = d[m] - d[l] + std::abs(e[l]) * cx(0.75, 0.25);   // exceptional shift
      cx s(1.0, 0.0), c(1.0, 0.0), p(0.0, 0.0);
      int i = m - 1;
      for (; i >= l; --i) {
        const cx f = s * e[i];
        const cx b = c * e[i];
        r = hyp(f, g);
        e[i + 1] = r;
        if (std::abs(r) <= 1e-300 + 1e-12 * (std::abs(f) + std::abs(g))) {
          if (std::abs(f) == 0.0 && std::abs(g) == 0.0) {   // exact split: deflate and restart
            d[i + 1] -= p;
            e[m] = 0.0;
            break;
          }
          return false;                                     // f = +-i g: the rotation breaks down
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
      }
      if (i >= l) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  for (const cx& z : d)
    if (!std::isfinite(z.real()) || !std::isfinite(z.imag())) return false;
  return true;
}

}  // namespace

extern "C" int ov_tridiag_eigenvalues(int32_t k, const double* alpha, const double* beta, const double* delta,
                                      double* eig) {
  if (k < 1 || !alpha || !delta || !eig || (k > 1 && !beta)) return OV_ERR_INVALID_ARG;
  std::vector<cx> d(k), e(k, cx(0.0, 0.0));
  for (int j = 0; j < k; ++j) d[j] = cx(alpha[2 * j], alpha[2 * j + 1]);
  for (int j = 0; j + 1 < k; ++j) e[j] = std::sqrt(cx(beta[2 * (j + 1)], beta[2 * (j + 1) + 1]) * delta[j + 1]);
  for (int j = 0; j < k; ++j)
    if (!std::isfinite(d[j].real()) || !std::isfinite(d[j].imag()) || !std::isfinite(e[j].real()) ||
        !std::isfinite(e[j].imag()))
      return OV_ERR_NONFINITE;
  if (!ql_complex_symmetric(d, e)) return OV_ERR_NOCONV;
  for (int j = 0; j < k; ++j) {
    eig[2 * j] = d[j].real();
    eig[2 * j + 1] = d[j].imag();
  }
  return OV_OK;
}

// Eigenvectors of T_k for a given (Ritz) eigenvalue theta, by inverse iteration
// (Wilkinson, "The Algebraic Eigenvalue Problem", ch. 9): three solves of
// (M - sigma) x = x with M = T_k (right eigenvector) or M = T_k^dag and
// sigma = conj(theta) (left eigenvector z, z^dag T_k = theta z^dag), each by
// Gaussian elimination with partial pivoting on the tridiagonal (rows exchanged
// as needed; the fill-in is one second superdiagonal).  A pivot that vanishes
// exactly is replaced by eps ||M||, which keeps the solve finite and leaves its
// direction that of the eigenvector.
namespace {

bool tridiag_solve(std::vector<cx> dl, std::vector<cx> d, std::vector<cx> du, std::vector<cx>& b, double tiny) {
  const int n = (int)d.size();
  std::vector<cx> du2(n > 2 ? n - 2 : 0, cx(0.0, 0.0));
  std::vector<char> swapped(n > 1 ? n - 1 : 0, 0);
  for (int i = 0; i + 1 < n; ++i) {
    if (std::abs(d[i]) >= std::abs(dl[i])) {
      if (d[i] == cx(0.0, 0.0)) d[i] = tiny;
      const cx f = dl[i] / d[i];
      dl[i] = f;
      d[i + 1] -= f * du[i];
    } else {
      const cx f = d[i] / dl[i];
      d[i] = dl[i];
      dl[i] = f;
      const cx t = du[i];
      du[i] = d[i + 1];
      d[i + 1] = t - f * d[i + 1];
      if (i + 2 < n) {
        du2[i] = du[i + 1];
        du[i + 1] = -f * du[i + 1];
      }
      swapped[i] = 1;
    }
  }
  if (d[n - 1] == cx(0.0, 0.0)) d[n - 1] = tiny;
  for (int i = 0; i + 1 < n; ++i) {
    if (swapped[i]) {
      const cx t = b[i];
      b[i] = b[i + 1];
      b[i + 1] = t - dl[i] * b[i];
    } else {
      b[i + 1] -= dl[i] * b[i];
    }
  }
  b[n - 1] /= d[n - 1];
  if (n > 1) b[n - 2] = (b[n - 2] - du[n - 2] * b[n - 1]) / d[n - 2];
  for (int i = n - 3; i >= 0; --i) b[i] = (b[i] - du[i] * b[i + 1] - du2[i] * b[i + 2]) / d[i];
  for (const cx& v : b)
    if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) return false;
  return true;
}

}  // namespace

extern "C" int ov_tridiag_eigenvector(int32_t k, const double* alpha, const double* beta, const double* delta,
                                      const double* theta, int32_t left, double* vec) {
  if (k < 1 || !alpha || !delta || !theta || !vec || (k > 1 && !beta) || (left != 0 && left != 1))
    return OV_ERR_INVALID_ARG;
  const cx th(theta[0], theta[1]);
  std::vector<cx> d(k), dl(k > 1 ? k - 1 : 0), du(k > 1 ? k - 1 : 0);
  double nrm = 0.0;
  for (int j = 0; j < k; ++j) {
    const cx a(alpha[2 * j], alpha[2 * j + 1]);
    d[j] = left ? std::conj(a) - std::conj(th) : a - th;
    nrm = std::max(nrm, std::abs(a));
  }
  for (int j = 1; j < k; ++j) {
    const cx b(beta[2 * j], beta[2 * j + 1]);   // T[j-1][j]
    const cx s(delta[j], 0.0);                  // T[j][j-1]
    du[j - 1] = left ? std::conj(s) : b;
    dl[j - 1] = left ? std::conj(b) : s;
    nrm = std::max(nrm, std::max(std::abs(b), std::abs(s)));
  }
  if (!std::isfinite(nrm) || !std::isfinite(th.real()) || !std::isfinite(th.imag())) return OV_ERR_NONFINITE;
  const double tiny = 2.220446049250313e-16 * (nrm > 0.0 ? nrm : 1.0);
  std::vector<cx> x(k, cx(1.0 / std::sqrt((double)k), 0.0));
  for (int it = 0; it < 3; ++it) {
    if (!tridiag_solve(dl, d, du, x, tiny)) return OV_ERR_NOCONV;
    double s = 0.0;
    for (const cx& v : x) s += std::norm(v);
    s = std::sqrt(s);
    if (!(s > 0.0) || !std::isfinite(s)) return OV_ERR_NOCONV;
    for (cx& v : x) v /= s;
  }
  for (int j = 0; j < k; ++j) {
    vec[2 * j] = x[j].real();
    vec[2 * j + 1] = x[j].imag();
  }
  return OV_OK;
}

// Eigenvalues and right eigenvectors of a small complex upper Hessenberg matrix (the
// Arnoldi matrix of the shift-and-invert eigen-solver), on the host: the implicit
// single-shift QR algorithm with Wilkinson shifts and exceptional shifts (Francis
// 1961-62; Golub and Van Loan, "Matrix Computations", ch. 7.5) for the eigenvalues,
// then inverse iteration on the original matrix with a pivoted LU for each
// eigenvector.  O(m^3); meant for m up to a few hundred.
namespace {

using cmat = std::vector<cx>;   // row-major m x m

bool hessenberg_qr(cmat t, int m, std::vector<cx>& eig) {
  const double eps = 2.220446049250313e-16;
  eig.assign(m, cx(0.0, 0.0));
  auto at = [&](int i, int j) -> cx& { return t[(size_t)i * m + j]; };
  int hi = m - 1, iter = 0, total = 0;
  while (hi >= 0) {
    if (hi == 0) {
      eig[0] = at(0, 0);
      break;
    }
    // the active block [lo, hi]: the first negligible subdiagonal above hi
    int lo = hi;
    while (lo > 0) {
      const double s = std::abs(at(lo, lo)) + std::abs(at(lo - 1, lo - 1));
      if (std::abs(at(lo, lo - 1)) <= eps * (s > 0.0 ? s : 1.0)) {
        at(lo, lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {
      eig[hi] = at(hi, hi);
      --hi;
      iter = 0;
      continue;
    }
    if (++total > 60 * m) return false;
    // Wilkinson shift from the trailing 2 x 2 block; an exceptional shift every 10
    cx sigma;
    if (++iter % 10 == 0) {
      sigma = at(hi, hi) + 0.75 * std::abs(at(hi, hi - 1));
    } else {
      const cx a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
      const cx tr2 = 0.5 * (a + d), det = a * d - b * c;
      const cx disc = std::sqrt(tr2 * tr2 - det);
      const cx e1 = tr2 + disc, e2 = tr2 - disc;
      sigma = std::abs(e1 - d) < std::abs(e2 - d) ? e1 : e2;
    }
    // implicit QR step on rows / columns lo..hi: the first rotation from the shifted
    // first column, then the bulge chased down the subdiagonal
    cx x = at(lo, lo) - sigma, y = at(lo + 1, lo);
    for (int k = lo; k < hi; ++k) {
      if (k > lo) {
        x = at(k, k - 1);
        y = at(k + 1, k - 1);
      }
      const double nr = std::sqrt(std::norm(x) + std::norm(y));
      if (nr == 0.0) continue;
      const cx cc = x / nr, ss = y / nr;   // G = [[conj c, conj s], [-s, c]] zeroes y
      const int c0 = k > lo ? k - 1 : lo;
      for (int j = c0; j <= hi; ++j) {     // rows k, k+1
        const cx p = at(k, j), q = at(k + 1, j);
        at(k, j) = std::conj(cc) * p + std::conj(ss) * q;
        at(k + 1, j) = -ss * p + cc * q;
      }
      const int r1 = std::min(k + 2, hi);
      for (int i = lo; i <= r1; ++i) {    // columns k, k+1 (G^dag from the right)
        const cx p = at(i, k), q = at(i, k + 1);
        at(i, k) = cc * p + ss * q;
        at(i, k + 1) = -std::conj(ss) * p + std::conj(cc) * q;
      }
      if (k > lo) at(k + 1, k - 1) = 0.0;
    }
  }
  return true;
}

// (A - mu) x = b by LU with partial pivoting (a zero pivot replaced by tiny)
bool dense_shift_solve(const cmat& a, int m, cx mu, std::vector<cx>& b, double tiny) {
  cmat w(a);
  for (int i = 0; i < m; ++i) w[(size_t)i * m + i] -= mu;
  for (int k = 0; k < m; ++k) {
    int p = k;
    for (int i = k + 1; i < m; ++i)
      if (std::abs(w[(size_t)i * m + k]) > std::abs(w[(size_t)p * m + k])) p = i;
    if (p != k) {
      for (int j = 0; j < m; ++j) std::swap(w[(size_t)k * m + j], w[(size_t)p * m + j]);
      std::swap(b[k], b[p]);
    }
    if (w[(size_t)k * m + k] == cx(0.0, 0.0)) w[(size_t)k * m + k] = tiny;
    for (int i = k + 1; i < m; ++i) {
      const cx f = w[(size_t)i * m + k] / w[(size_t)k * m + k];
      if (f == cx(0.0, 0.0)) continue;
      for (int j = k; j < m; ++j) w[(size_t)i * m + j] -= f * w[(size_t)k * m + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    cx s = b[i];
    for (int j = i + 1; j < m; ++j) s -= w[(size_t)i * m + j] * b[j];
    b[i] = s / w[(size_t)i * m + i];
  }
  for (const cx& v : b)
    if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) return false;
  return true;
}

}  // namespace

extern "C" int ov_hessenberg_eigen(int32_t m, const double* h, double* eig, double* vecs) {
  if (m < 1 || m > 4096 || !h || !eig) return OV_ERR_INVALID_ARG;
  cmat a((size_t)m * m);
  double nrm = 0.0;
  for (size_t i = 0; i < a.size(); ++i) {
    a[i] = cx(h[2 * i], h[2 * i + 1]);
    if (!std::isfinite(h[2 * i]) || !std::isfinite(h[2 * i + 1])) return OV_ERR_NONFINITE;
    nrm = std::max(nrm, std::abs(a[i]));
  }
  for (int i = 2; i < m; ++i)
    for (int j = 0; j < i - 1; ++j)
      if (a[(size_t)i * m + j] != cx(0.0, 0.0)) return OV_ERR_INVALID_ARG;   // not upper Hessenberg
  std::vector<cx> ev;
  if (!hessenberg_qr(a, m, ev)) return OV_ERR_NOCONV;
  const double tiny = 2.220446049250313e-16 * (nrm > 0.0 ? nrm : 1.0);
  for (int i = 0; i < m; ++i) {
    eig[2 * i] = ev[i].real();
    eig[2 * i + 1] = ev[i].imag();
    if (!vecs) continue;
    std::vector<cx> x(m, cx(1.0 / std::sqrt((double)m), 0.0));
    for (int it = 0; it < 3; ++it) {
      if (!dense_shift_solve(a, m, ev[i], x, tiny)) return OV_ERR_NOCONV;
      double s = 0.0;
      for (const cx& v : x) s += std::norm(v);
      s = std::sqrt(s);
      if (!(s > 0.0) || !std::isfinite(s)) return OV_ERR_NOCONV;
      for (cx& v : x) v /= s;
    }
    for (int j = 0; j < m; ++j) {      // column i of vecs (row-major m x m)
      vecs[2 * ((size_t)j * m + i)] = x[j].real();
      vecs[2 * ((size_t)j * m + i) + 1] = x[j].imag();
    }
  }
  return OV_OK;
}
