// Host-only entry points over the FP64 host numerics of the block GMRES
// (paper_2008_01966_gb300/csrc/bgmres_host.h), built with g++ by
// tests/test_block_host.py for CPU tests.  Complex arrays are interleaved
// (re, im) doubles, row-major.
#include <cstring>

#include "bgmres_host.h"

static std::vector<cd> load(const double* p, size_t n) {
  return std::vector<cd>((const cd*)p, (const cd*)p + n);
}

extern "C" {

void shim_herm_eig(const double* a, int n, double* lam, double* U) {
  std::vector<double> l;
  std::vector<cd> u;
  herm_eig(load(a, (size_t)n * n), n, l, u);
  std::memcpy(lam, l.data(), sizeof(double) * n);
  std::memcpy(U, u.data(), sizeof(cd) * n * n);
}

// T: n x BG_MAX, S: n x n; returns 1 when the factorisation was accepted
int shim_cholqr(const double* G, int n, double* T, double* S, double* cond) {
  std::vector<cd> t, s;
  double c = 0;
  const bool ok = cholqr(load(G, (size_t)n * n), n, t, s, c);
  if (ok) {
    std::memcpy(T, t.data(), sizeof(cd) * n * BG_MAX);
    std::memcpy(S, s.data(), sizeof(cd) * n * n);
  }
  *cond = c;
  return ok ? 1 : 0;
}

double shim_svqb(const double* G, int n, double* T, double* S, double* ratio) {
  std::vector<cd> t, s;
  const double dev = svqb(load(G, (size_t)n * n), n, t, s, *ratio);
  std::memcpy(T, t.data(), sizeof(cd) * n * BG_MAX);
  std::memcpy(S, s.data(), sizeof(cd) * n * n);
  return dev;
}

void shim_matmul_left(const double* S2, double* S, int n) {
  std::vector<cd> s = load(S, (size_t)n * n);
  matmul_left(load(S2, (size_t)n * n), s, n);
  std::memcpy(S, s.data(), sizeof(cd) * n * n);
}

// Least squares min || E_1 S0 - Hbar Y || for a block upper Hessenberg Hbar of
// nblk block columns of width r ((nblk + 1) r rows, row-major, leading
// dimension nblk r), added one block column at a time.  res[k r + j]: residual
// of right-hand side j after block column k; Y: nblk r x r.
void shim_blockls(int r, const double* S0, int nblk, const double* Hbar, double* Y, double* res) {
  const cd* H = (const cd*)Hbar;
  const int ld = nblk * r;
  BlockLS ls;
  ls.start(r, load(S0, (size_t)r * r));
  for (int k = 0; k < nblk; ++k) {
    const int rows = (k + 2) * r;
    std::vector<std::vector<cd>> cols(r, std::vector<cd>(rows));
    for (int j = 0; j < r; ++j)
      for (int i = 0; i < rows; ++i) cols[j][i] = H[(size_t)i * ld + k * r + j];
    ls.add(cols, rows);
    for (int j = 0; j < r; ++j) res[k * r + j] = ls.resid(j);
  }
  std::vector<cd> y;
  ls.solve(y);
  cd* out = (cd*)Y;
  for (int i = 0; i < nblk * r; ++i)
    for (int j = 0; j < r; ++j) out[(size_t)i * r + j] = y[(size_t)i * BG_MAX + j];
}
}
