// Host-side numerics of the FP32 block GMRES (bgmres.cu), in FP64: the
// Hermitian eigendecomposition behind SVQB, the Cholesky QR and SVQB steps
// that orthonormalise a new block from its Gram matrix, and the Householder
// least-squares solve of the block upper Hessenberg system.  Plain C++ (no
// CUDA), so the same code also builds on its own for host-only tests.
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#define BG_MAX 16  // directions per group (columns of a block)

typedef std::complex<double> cd;

// Eigendecomposition of a Hermitian n x n matrix (row-major) by cyclic Jacobi
// rotations: a = U diag(lam) U^H.  The rotation for entry (p, q) is computed
// from t = tan(theta) of the 2 x 2 problem without trigonometric calls.
static void herm_eig(std::vector<cd> a, int n, std::vector<double>& lam, std::vector<cd>& U) {
  U.assign((size_t)n * n, cd(0, 0));
  for (int i = 0; i < n; ++i) U[(size_t)i * n + i] = 1.0;
  auto A = [&](int i, int j) -> cd& { return a[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0, dia = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? dia : off) += std::norm(A(i, j));
    if (off <= 1e-30 * std::max(dia, 1e-300)) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const cd apq = A(p, q);
        const double m2 = std::norm(apq);
        if (m2 <= 1e-34 * std::abs(A(p, p).real() * A(q, q).real()) || m2 == 0.0) continue;
        const double m = std::sqrt(m2);
        const cd ph = apq / m;
        // zero the (p, q) entry: tan(2 theta) = 2 m / (a_qq - a_pp), |theta| <= pi/4
        const double tau = (A(q, q).real() - A(p, p).real()) / (2 * m);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        // J: columns p, q of the identity replaced by (c, -s conj(ph)) and (s ph, c)
        const cd jpq = s * ph, jqp = -s * std::conj(ph);
        for (int k = 0; k < n; ++k) {  // a <- a J
          const cd x = A(k, p), y = A(k, q);
          A(k, p) = x * c + y * jqp;
          A(k, q) = x * jpq + y * c;
        }
        for (int k = 0; k < n; ++k) {  // a <- J^H a
          const cd x = A(p, k), y = A(q, k);
          A(p, k) = c * x + std::conj(jqp) * y;
          A(q, k) = std::conj(jpq) * x + c * y;
        }
        A(p, q) = A(q, p) = 0.0;
        A(p, p) = A(p, p).real();
        A(q, q) = A(q, q).real();
        for (int k = 0; k < n; ++k) {  // U <- U J
          const cd x = U[(size_t)k * n + p], y = U[(size_t)k * n + q];
          U[(size_t)k * n + p] = x * c + y * jqp;
          U[(size_t)k * n + q] = x * jpq + y * c;
        }
      }
    }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = A(i, i).real();
}

// Cholesky QR step: G = L L^H, T = L^{-H} (the block transform, BG_MAX wide),
// S = L^H (old block = new block * S).  Returns false when a pivot falls below
// 1e-10 of the largest diagonal entry; cond receives an upper bound of the
// condition number of G, ||G||_F ||L^{-1}||_F^2.
static bool cholqr(const std::vector<cd>& G, int n, std::vector<cd>& T, std::vector<cd>& S,
                   double& cond) {
  std::vector<cd> L((size_t)n * n, cd(0, 0));
  double dmax = 0, gf = 0;
  for (int i = 0; i < n; ++i) dmax = std::max(dmax, G[(size_t)i * n + i].real());
  for (const cd& x : G) gf += std::norm(x);
  if (!(dmax > 0)) return false;
  for (int j = 0; j < n; ++j) {
    double d = G[(size_t)j * n + j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(L[(size_t)j * n + k]);
    if (!(d > 1e-10 * dmax)) return false;
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      cd v = G[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * std::conj(L[(size_t)j * n + k]);
      L[(size_t)i * n + j] = v / ljj;
    }
  }
  // Li = L^{-1} (lower triangular)
  std::vector<cd> Li((size_t)n * n, cd(0, 0));
  for (int c = 0; c < n; ++c) {
    Li[(size_t)c * n + c] = 1.0 / L[(size_t)c * n + c];
    for (int i = c + 1; i < n; ++i) {
      cd v = 0;
      for (int k = c; k < i; ++k) v -= L[(size_t)i * n + k] * Li[(size_t)k * n + c];
      Li[(size_t)i * n + c] = v / L[(size_t)i * n + i];
    }
  }
  double lf = 0;
  for (const cd& x : Li) lf += std::norm(x);
  cond = std::sqrt(gf) * lf;
  T.assign((size_t)n * BG_MAX, cd(0, 0));
  S.assign((size_t)n * n, cd(0, 0));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      T[(size_t)i * BG_MAX + j] = std::conj(Li[(size_t)j * n + i]);  // (L^{-1})^H
      S[(size_t)i * n + j] = std::conj(L[(size_t)j * n + i]);        // L^H
    }
  return true;
}

// One SVQB step on the Gram matrix G (n x n): T = U Lambda_c^{-1/2} (the
// transform of the block, stored BG_MAX wide as the k_bnn_tc5 coefficient matrix),
// S = Lambda_c^{1/2} U^H (W = (W T) S); Lambda_c = max(Lambda, floor).
// Returns the deviation of G from the identity (max |G - I|); ratio receives
// min(Lambda) / max(Lambda).
static double svqb(const std::vector<cd>& G, int n, std::vector<cd>& T, std::vector<cd>& S,
                   double& ratio) {
  double dev = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) dev = std::max(dev, std::abs(G[(size_t)i * n + j] - (i == j ? 1.0 : 0.0)));
  std::vector<double> lam;
  std::vector<cd> U;
  herm_eig(G, n, lam, U);
  double lmax = 0, lmin = 1e300;
  for (double l : lam) {
    lmax = std::max(lmax, l);
    lmin = std::min(lmin, l);
  }
  ratio = lmax > 0 ? lmin / lmax : 0.0;
  T.assign((size_t)n * BG_MAX, cd(0, 0));
  S.assign((size_t)n * n, cd(0, 0));
  if (!(lmax > 1e-300)) return dev;  // the block vanished (exact breakdown): zero block
  const double fl = lmax * 1e-12;
  for (int c = 0; c < n; ++c) {
    const double l = std::max(lam[c], fl), sl = std::sqrt(l);
    for (int i = 0; i < n; ++i) {
      T[(size_t)i * BG_MAX + c] = U[(size_t)i * n + c] / sl;
      S[(size_t)c * n + i] = sl * std::conj(U[(size_t)i * n + c]);
    }
  }
  return dev;
}

// S <- S2 S  (n x n, row-major)
static void matmul_left(const std::vector<cd>& S2, std::vector<cd>& S, int n) {
  std::vector<cd> o((size_t)n * n, cd(0, 0));
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const cd a = S2[(size_t)i * n + k];
      for (int j = 0; j < n; ++j) o[(size_t)i * n + j] += a * S[(size_t)k * n + j];
    }
  S.swap(o);
}

// Householder QR of the block Hessenberg matrix of one group, one column at a time.
struct BlockLS {
  int r = 0;                         // block width = right-hand sides
  int rows = 0, cols = 0;            // current size of Hbar
  std::vector<std::vector<cd>> v;    // reflector c acts on rows c .. c + v[c].size() - 1
  std::vector<std::vector<cd>> R;    // column c of the triangular factor (rows 0..c)
  std::vector<cd> g;                 // rows x r transformed right-hand sides (row-major)
  void start(int r_, const std::vector<cd>& S0) {
    r = r_;
    rows = r;
    cols = 0;
    v.clear();
    R.clear();
    g = S0;
  }
  // append block column: col[c] has rows_new entries (rows 0..rows_new-1)
  void add(const std::vector<std::vector<cd>>& newcols, int rows_new) {
    g.resize((size_t)rows_new * r, cd(0, 0));
    rows = rows_new;
    // the reflectors so far, each applied to all new columns at once
    std::vector<std::vector<cd>> nc(newcols.size());
    for (size_t c = 0; c < newcols.size(); ++c) {
      nc[c] = newcols[c];
      nc[c].resize(rows, cd(0, 0));
    }
    for (int p = 0; p < cols; ++p) {
      const auto& vp = v[p];
      const size_t L = vp.size();
      for (auto& col : nc) {
        cd* x = col.data() + p;
        double sr = 0, si = 0;
        for (size_t t = 0; t < L; ++t) {  // s = v^H x
          sr += vp[t].real() * x[t].real() + vp[t].imag() * x[t].imag();
          si += vp[t].real() * x[t].imag() - vp[t].imag() * x[t].real();
        }
        sr *= 2;
        si *= 2;
        for (size_t t = 0; t < L; ++t)  // x -= 2 v s
          x[t] -= cd(vp[t].real() * sr - vp[t].imag() * si, vp[t].real() * si + vp[t].imag() * sr);
      }
    }
    for (size_t cix = 0; cix < nc.size(); ++cix) {
      std::vector<cd>& col = nc[cix];
      // reflectors of the earlier new columns of this block
      for (int p = cols - (int)cix; p < cols; ++p) {
        const auto& vp = v[p];
        cd s = 0;
        for (size_t t = 0; t < vp.size(); ++t) s += std::conj(vp[t]) * col[p + t];
        for (size_t t = 0; t < vp.size(); ++t) col[p + t] -= 2.0 * vp[t] * s;
      }
      const int ci = cols;
      double alpha = 0;
      for (int t = ci; t < rows; ++t) alpha += std::norm(col[t]);
      alpha = std::sqrt(alpha);
      const double a0 = std::abs(col[ci]);
      const cd ph = a0 > 0 ? col[ci] / a0 : cd(1, 0);
      std::vector<cd> u(col.begin() + ci, col.end());
      u[0] += ph * alpha;
      double un = 0;
      for (const cd& x : u) un += std::norm(x);
      un = std::sqrt(un);
      if (un > 0)
        for (cd& x : u) x /= un;
      for (int t = ci; t < rows; ++t) col[t] = 0;
      col[ci] = -ph * alpha;
      R.emplace_back(col.begin(), col.begin() + ci + 1);
      for (int j = 0; j < r; ++j) {
        cd s = 0;
        for (size_t t = 0; t < u.size(); ++t) s += std::conj(u[t]) * g[(size_t)(ci + t) * r + j];
        for (size_t t = 0; t < u.size(); ++t) g[(size_t)(ci + t) * r + j] -= 2.0 * u[t] * s;
      }
      v.push_back(std::move(u));
      ++cols;
    }
  }
  double resid(int j) const {
    double s = 0;
    for (int t = cols; t < rows; ++t) s += std::norm(g[(size_t)t * r + j]);
    return std::sqrt(s);
  }
  // Y = R^{-1} g[0:cols]  (cols x r, stored BG_MAX wide)
  void solve(std::vector<cd>& Y) const {
    Y.assign((size_t)cols * BG_MAX, cd(0, 0));
    for (int j = 0; j < r; ++j) {
      for (int i = cols - 1; i >= 0; --i) {
        cd s = g[(size_t)i * r + j];
        for (int k = i + 1; k < cols; ++k) s -= R[k][i] * Y[(size_t)k * BG_MAX + j];
        const cd d = R[i][i];
        Y[(size_t)i * BG_MAX + j] = std::abs(d) > 0 ? s / d : cd(0, 0);
      }
    }
  }
};
