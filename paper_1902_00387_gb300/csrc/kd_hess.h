// Small dense eigenproblem of the Arnoldi method (kd_arnoldi.cu, kd_hessenberg_eig):
// complex Schur form of an upper Hessenberg matrix by the shifted QR algorithm and the
// eigenvectors from it.  Host code only.
#pragma once

#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

namespace kd {
namespace hess {

using cd = std::complex<double>;

// Complex Schur form T = Q^H H Q of an upper Hessenberg m x m matrix (row-major, T
// overwrites H) by the shifted QR algorithm: Givens rotations, Wilkinson shifts, an
// exceptional shift every 10 iterations without deflation, deflation on negligible
// subdiagonal entries.  false if it did not converge.
inline bool hessenberg_schur(std::vector<cd>& H, std::vector<cd>& Q, int m) {
  Q.assign((size_t)m * m, cd(0.0));
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  auto at = [&](int i, int j) -> cd& { return H[(size_t)i * m + j]; };
  const double eps = 1e-15;
  int hi = m - 1, iter = 0, total = 0;
  std::vector<cd> cs(m), sn(m);
  while (hi > 0) {
    if (++total > 100 * m) return false;
    int l = hi;
    while (l > 0 && std::abs(at(l, l - 1)) > eps * (std::abs(at(l - 1, l - 1)) + std::abs(at(l, l)))) --l;
    if (l > 0) at(l, l - 1) = 0.0;
    if (l == hi) {
      --hi;
      iter = 0;
      continue;
    }
    // shift: eigenvalue of the trailing 2 x 2 block closer to its last diagonal entry
    const cd a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
    const cd tr = a + d, det = a * d - b * c;
    const cd disc = std::sqrt(tr * tr / 4.0 - det);
    const cd m1 = tr / 2.0 + disc, m2 = tr / 2.0 - disc;
    cd mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
    if (iter % 10 == 9) mu = d + std::abs(c);
    ++iter;
    for (int k = l; k <= hi; ++k) at(k, k) -= mu;
    // H - mu I = G R: row rotations zero the subdiagonal of the active block
    for (int k = l; k < hi; ++k) {
      const cd x = at(k, k), y = at(k + 1, k);
      const double r = std::sqrt(std::norm(x) + std::norm(y));
      cs[k] = r > 0 ? x / r : cd(1.0);
      sn[k] = r > 0 ? y / r : cd(0.0);
      for (int j = k; j < m; ++j) {
        const cd u = at(k, j), v = at(k + 1, j);
        at(k, j) = std::conj(cs[k]) * u + std::conj(sn[k]) * v;
        at(k + 1, j) = -sn[k] * u + cs[k] * v;
      }
    }
    // R G + mu I, and Q <- Q G
    for (int k = l; k < hi; ++k) {
      for (int i = 0; i <= std::min(k + 1, hi); ++i) {
        const cd u = at(i, k), v = at(i, k + 1);
        at(i, k) = u * cs[k] + v * sn[k];
        at(i, k + 1) = -u * std::conj(sn[k]) + v * std::conj(cs[k]);
      }
      for (int i = 0; i < m; ++i) {
        const cd u = Q[(size_t)i * m + k], v = Q[(size_t)i * m + k + 1];
        Q[(size_t)i * m + k] = u * cs[k] + v * sn[k];
        Q[(size_t)i * m + k + 1] = -u * std::conj(sn[k]) + v * std::conj(cs[k]);
      }
    }
    for (int k = l; k <= hi; ++k) at(k, k) += mu;
  }
  return true;
}

// unit eigenvector of H for the eigenvalue T[p][p] of its Schur form: y = Q z, T z = T_pp z
inline std::vector<cd> schur_vector(const std::vector<cd>& T, const std::vector<cd>& Q, int m, int p) {
  std::vector<cd> z(m, cd(0.0));
  z[p] = 1.0;
  const cd lam = T[(size_t)p * m + p];
  const double small = 1e-14 * std::max(1.0, std::abs(lam));
  for (int i = p - 1; i >= 0; --i) {
    cd s = 0.0;
    for (int j = i + 1; j <= p; ++j) s += T[(size_t)i * m + j] * z[j];
    cd den = T[(size_t)i * m + i] - lam;
    if (std::abs(den) < small) den = small;
    z[i] = -s / den;
  }
  std::vector<cd> y(m, cd(0.0));
  double nrm = 0.0;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j <= p; ++j) y[i] += Q[(size_t)i * m + j] * z[j];
    nrm += std::norm(y[i]);
  }
  nrm = std::sqrt(nrm);
  for (auto& v : y) v /= nrm;
  return y;
}

}  // namespace hess
}  // namespace kd
