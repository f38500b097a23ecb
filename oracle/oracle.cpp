// FP64 CPU oracle of the CPR-FGMRES black-oil Jacobian solver.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark may load this library; the solver itself
// never calls it.  It shares no code with the GPU path.  Every routine is
// the plain definition (or the paper's algorithm step by step), single
// threaded, in double precision, written for a reader to check by eye:
//
//   or_bsr_spmv            y = A x                     (Sec. 3.3, y = alpha A x + beta y)
//   or_qi_decouple         D_QI^{-1} A                 (Sec. 3.2, Quasi-IMPES operator)
//   or_bsr_permute         P A P^T                     (orderings for ILU(0))
//   or_bsr_ilu0 / _solve   block ILU(0), IKJ form      (Sec. 3.2, RAS local solver ILU(0))
//   or_dense_solve         dense LU, partial pivoting  (pins and coarse solves)
//   or_amg_*               aggregation AMG V-cycle on A_pp   (Sec. 3.2, Alg. 2 "AMG(A_pp)")
//   or_cpr_*               CPR-FPF                     (Sec. 3.2, Alg. 2)
//   or_gmres               restarted right-preconditioned GMRES(m), MGS
//                                                       (Sec. 3.3 solver list; GMRES(30) in Sec. 4)
//   or_bicgstab            right-preconditioned BiCGSTAB (Sec. 3.3 solver list; the
//                                                       solver of Sec. 4's scalability runs)
//   or_rel_residual        ||b - A x|| / ||b||, compensated sums (Alg. 1 criterion)
//   or_bsr_spmv_threads    y = A x over T host threads: the CPU bandwidth
//                          baseline of the benchmark (the only threaded routine)
//
// Layout conventions: BSR with bs x bs blocks stored row-major inside a
// block; block columns sorted ascending within a block row.  Unknown k of
// block row i is entry bs*i + k of a vector.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <thread>
#include <vector>

namespace {

constexpr int kOk = 0;
constexpr int kBreakdown = -6;
constexpr int kNotConverged = -7;
constexpr int kArg = -1;

// ---------------------------------------------------------------- small dense
// Solve M x = r for one bs x bs block by Gaussian elimination with partial
// pivoting.  Returns false on an exactly zero pivot.
bool block_solve(int bs, const double* M, const double* r, double* x) {
  double a[8][8], b[8];
  for (int i = 0; i < bs; ++i) {
    b[i] = r[i];
    for (int j = 0; j < bs; ++j) a[i][j] = M[bs * i + j];
  }
  for (int k = 0; k < bs; ++k) {
    int p = k;
    for (int i = k + 1; i < bs; ++i)
      if (std::fabs(a[i][k]) > std::fabs(a[p][k])) p = i;
    if (a[p][k] == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < bs; ++j) std::swap(a[k][j], a[p][j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < bs; ++i) {
      const double l = a[i][k] / a[k][k];
      for (int j = k; j < bs; ++j) a[i][j] -= l * a[k][j];
      b[i] -= l * b[k];
    }
  }
  for (int i = bs - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < bs; ++j) s -= a[i][j] * x[j];
    x[i] = s / a[i][i];
  }
  return true;
}

// C = A * B for bs x bs blocks
void block_mul(int bs, const double* A, const double* B, double* C) {
  for (int i = 0; i < bs; ++i)
    for (int j = 0; j < bs; ++j) {
      double s = 0;
      for (int k = 0; k < bs; ++k) s += A[bs * i + k] * B[bs * k + j];
      C[bs * i + j] = s;
    }
}

// X = B * inv(U): solve X U = B row by row (X^T = U^{-T} B^T)
bool block_right_div(int bs, const double* B, const double* U, double* X) {
  double Ut[64], row[8], sol[8];
  for (int i = 0; i < bs; ++i)
    for (int j = 0; j < bs; ++j) Ut[bs * i + j] = U[bs * j + i];
  for (int i = 0; i < bs; ++i) {
    for (int j = 0; j < bs; ++j) row[j] = B[bs * i + j];
    if (!block_solve(bs, Ut, row, sol)) return false;
    for (int j = 0; j < bs; ++j) X[bs * i + j] = sol[j];
  }
  return true;
}

struct Bsr {
  int64_t nb = 0;
  int bs = 3;
  std::vector<int32_t> rowptr, col;
  std::vector<double> val;
  void spmv(const double* x, double* y) const {
    for (int64_t i = 0; i < nb; ++i) {
      for (int r = 0; r < bs; ++r) {
        double s = 0;
        for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
          for (int c = 0; c < bs; ++c) s += val[(size_t)e * bs * bs + bs * r + c] * x[(size_t)col[e] * bs + c];
        y[i * bs + r] = s;
      }
    }
  }
  int64_t n() const { return nb * bs; }
};

Bsr make_bsr(int64_t nb, int bs, const int32_t* rowptr, const int32_t* col, const double* val) {
  Bsr A;
  A.nb = nb;
  A.bs = bs;
  A.rowptr.assign(rowptr, rowptr + nb + 1);
  A.col.assign(col, col + rowptr[nb]);
  A.val.assign(val, val + (size_t)rowptr[nb] * bs * bs);
  return A;
}

double dot(int64_t n, const double* a, const double* b) {
  double s = 0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

// ---------------------------------------------------------------- block ILU(0)
// ILU(0) of a BSR matrix in its given ordering (IKJ form).  On return lu
// holds L (unit lower, strictly lower blocks) and U (upper blocks incl. the
// diagonal) on the pattern of A: for every (i, j) of the pattern,
// (L U)_ij = A_ij.
int ilu0_factor(const Bsr& A, std::vector<double>& lu) {
  const int bs = A.bs, b2 = bs * bs;
  lu = A.val;
  std::vector<int32_t> diag(A.nb, -1);
  for (int64_t i = 0; i < A.nb; ++i)
    for (int32_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e)
      if (A.col[e] == i) diag[i] = e;
  for (int64_t i = 0; i < A.nb; ++i)
    if (diag[i] < 0) return kBreakdown;
  std::vector<double> tmp(b2);
  for (int64_t i = 0; i < A.nb; ++i) {
    for (int32_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      const int64_t k = A.col[e];
      if (k >= i) break;  // columns ascending: only the strictly lower part
      // L_ik = A_ik U_kk^{-1}
      if (!block_right_div(bs, &lu[(size_t)e * b2], &lu[(size_t)diag[k] * b2], tmp.data())) return kBreakdown;
      std::copy(tmp.begin(), tmp.end(), lu.begin() + (size_t)e * b2);
      // A_ij -= L_ik U_kj for j > k on the pattern of row i
      for (int32_t f = e + 1; f < A.rowptr[i + 1]; ++f) {
        const int64_t j = A.col[f];
        for (int32_t g = A.rowptr[k]; g < A.rowptr[k + 1]; ++g) {
          if (A.col[g] != j) continue;
          double prod[64];
          block_mul(bs, &lu[(size_t)e * b2], &lu[(size_t)g * b2], prod);
          for (int t = 0; t < b2; ++t) lu[(size_t)f * b2 + t] -= prod[t];
        }
      }
    }
    // the pivot block must be invertible
    std::vector<double> probe(bs, 0.0), sol(bs);
    probe[0] = 1.0;
    if (!block_solve(bs, &lu[(size_t)diag[i] * b2], probe.data(), sol.data())) return kBreakdown;
  }
  return kOk;
}

// z = (L U)^{-1} r
void ilu0_solve(const Bsr& A, const std::vector<double>& lu, const double* r, double* z) {
  const int bs = A.bs, b2 = bs * bs;
  std::vector<double> y(A.n());
  for (int64_t i = 0; i < A.nb; ++i) {  // L y = r, unit diagonal
    for (int c = 0; c < bs; ++c) y[i * bs + c] = r[i * bs + c];
    for (int32_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      const int64_t k = A.col[e];
      if (k >= i) break;
      for (int rr = 0; rr < bs; ++rr)
        for (int c = 0; c < bs; ++c) y[i * bs + rr] -= lu[(size_t)e * b2 + bs * rr + c] * y[k * bs + c];
    }
  }
  for (int64_t i = A.nb - 1; i >= 0; --i) {  // U z = y
    double s[8];
    int32_t d = -1;
    for (int c = 0; c < bs; ++c) s[c] = y[i * bs + c];
    for (int32_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      const int64_t k = A.col[e];
      if (k == i) { d = e; continue; }
      if (k < i) continue;
      for (int rr = 0; rr < bs; ++rr)
        for (int c = 0; c < bs; ++c) s[rr] -= lu[(size_t)e * b2 + bs * rr + c] * z[k * bs + c];
    }
    block_solve(bs, &lu[(size_t)d * b2], s, &z[i * bs]);
  }
}

// B = P A P^T with perm[new] = old; block columns of B sorted.
Bsr permute(const Bsr& A, const int64_t* perm) {
  Bsr B;
  B.nb = A.nb;
  B.bs = A.bs;
  const int b2 = A.bs * A.bs;
  std::vector<int64_t> inv(A.nb);
  for (int64_t i = 0; i < A.nb; ++i) inv[perm[i]] = i;
  B.rowptr.assign(A.nb + 1, 0);
  B.col.reserve(A.col.size());
  B.val.reserve(A.val.size());
  for (int64_t ni = 0; ni < A.nb; ++ni) {
    const int64_t oi = perm[ni];
    std::vector<std::pair<int64_t, int32_t>> row;
    for (int32_t e = A.rowptr[oi]; e < A.rowptr[oi + 1]; ++e) row.push_back({inv[A.col[e]], e});
    std::sort(row.begin(), row.end());
    for (auto& p : row) {
      B.col.push_back((int32_t)p.first);
      B.val.insert(B.val.end(), A.val.begin() + (size_t)p.second * b2, A.val.begin() + (size_t)(p.second + 1) * b2);
    }
    B.rowptr[ni + 1] = (int32_t)B.col.size();
  }
  return B;
}

// ---------------------------------------------------------------- dense LU
struct DenseLU {
  int n = 0;
  std::vector<double> a;
  std::vector<int> piv;
  int factor(int n_, const double* A) {
    n = n_;
    a.assign(A, A + (size_t)n * n);
    piv.resize(n);
    for (int k = 0; k < n; ++k) {
      int p = k;
      for (int i = k + 1; i < n; ++i)
        if (std::fabs(a[(size_t)i * n + k]) > std::fabs(a[(size_t)p * n + k])) p = i;
      piv[k] = p;
      if (a[(size_t)p * n + k] == 0.0) return kBreakdown;
      if (p != k)
        for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
      for (int i = k + 1; i < n; ++i) {
        const double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
        a[(size_t)i * n + k] = l;
        for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
      }
    }
    return kOk;
  }
  void solve(const double* b, double* x) const {
    std::vector<double> y(b, b + n);
    for (int k = 0; k < n; ++k) std::swap(y[k], y[piv[k]]);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j) y[i] -= a[(size_t)i * n + j] * y[j];
    for (int i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int j = i + 1; j < n; ++j) s -= a[(size_t)i * n + j] * x[j];
      x[i] = s / a[(size_t)i * n + i];
    }
  }
};

// ---------------------------------------------------------------- AMG
// Aggregation AMG on a scalar matrix that lives on a structured nx x ny x nz
// grid (the pressure block A_pp).  Aggregates are the 2x2x2 boxes of cells
// (i/2, j/2, k/2); the prolongation P is piecewise constant (P_ic = 1 if
// cell i lies in aggregate c); the coarse operator is Galerkin A_c = P^T A P.
// Coarsening stops once a level has at most `coarse_max` cells or no axis
// can be halved; the coarsest level is solved by dense LU.
struct Csr {
  int64_t n = 0;
  std::vector<int32_t> rowptr, col;
  std::vector<double> val;
};

struct AmgLevel {
  int nx, ny, nz;
  Csr A;
  std::vector<int64_t> agg;  // fine cell -> coarse cell (empty on the coarsest level)
};

struct AmgParams {
  int smoother = 0;     // 0 red-black Gauss-Seidel, 1 damped Jacobi
  int nu1 = 1, nu2 = 1; // pre / post sweeps
  double omega = 0.6667;
  double overcorr = 1.0;  // coarse-correction scale s: x += s P x_c
  int coarse_max = 512;
  int max_levels = 20;
};

struct Amg {
  AmgParams prm;
  std::vector<AmgLevel> lv;
  DenseLU coarse;

  int setup(const Csr& A0, int nx, int ny, int nz, const AmgParams& p) {
    prm = p;
    lv.clear();
    lv.push_back(AmgLevel{nx, ny, nz, A0, {}});
    while ((int)lv.size() < prm.max_levels) {
      AmgLevel& f = lv.back();
      if (f.A.n <= prm.coarse_max) break;
      if (f.nx == 1 && f.ny == 1 && f.nz == 1) break;
      const int cx = (f.nx + 1) / 2, cy = (f.ny + 1) / 2, cz = (f.nz + 1) / 2;
      f.agg.resize(f.A.n);
      for (int k = 0; k < f.nz; ++k)
        for (int j = 0; j < f.ny; ++j)
          for (int i = 0; i < f.nx; ++i)
            f.agg[i + (int64_t)f.nx * (j + (int64_t)f.ny * k)] = i / 2 + (int64_t)cx * (j / 2 + (int64_t)cy * (k / 2));
      // Galerkin product A_c = P^T A P: entry a_ij adds to (agg i, agg j)
      const int64_t nc = (int64_t)cx * cy * cz;
      std::vector<std::map<int64_t, double>> rows(nc);
      for (int64_t i = 0; i < f.A.n; ++i)
        for (int32_t e = f.A.rowptr[i]; e < f.A.rowptr[i + 1]; ++e)
          rows[f.agg[i]][f.agg[f.A.col[e]]] += f.A.val[e];
      Csr C;
      C.n = nc;
      C.rowptr.assign(nc + 1, 0);
      for (int64_t i = 0; i < nc; ++i) {
        for (auto& kv : rows[i]) { C.col.push_back((int32_t)kv.first); C.val.push_back(kv.second); }
        C.rowptr[i + 1] = (int32_t)C.col.size();
      }
      lv.push_back(AmgLevel{cx, cy, cz, C, {}});
    }
    const Csr& Ac = lv.back().A;
    std::vector<double> dense((size_t)Ac.n * Ac.n, 0.0);
    for (int64_t i = 0; i < Ac.n; ++i)
      for (int32_t e = Ac.rowptr[i]; e < Ac.rowptr[i + 1]; ++e) dense[(size_t)i * Ac.n + Ac.col[e]] += Ac.val[e];
    return coarse.factor((int)Ac.n, dense.data());
  }

  static int color(const AmgLevel& L, int64_t c) {
    const int64_t i = c % L.nx, j = (c / L.nx) % L.ny, k = c / ((int64_t)L.nx * L.ny);
    return (int)((i + j + k) & 1);
  }

  // one Gauss-Seidel half sweep over the cells of colour `col`
  void gs_half(const AmgLevel& L, int col, const double* f, double* x) const {
    for (int64_t i = 0; i < L.A.n; ++i) {
      if (color(L, i) != col) continue;
      double s = f[i], d = 0;
      for (int32_t e = L.A.rowptr[i]; e < L.A.rowptr[i + 1]; ++e) {
        if (L.A.col[e] == i) d = L.A.val[e];
        else s -= L.A.val[e] * x[L.A.col[e]];
      }
      x[i] = s / d;
    }
  }

  void jacobi(const AmgLevel& L, const double* f, double* x) const {
    std::vector<double> xn(L.A.n);
    for (int64_t i = 0; i < L.A.n; ++i) {
      double s = f[i], d = 0;
      for (int32_t e = L.A.rowptr[i]; e < L.A.rowptr[i + 1]; ++e) {
        s -= L.A.val[e] * x[L.A.col[e]];
        if (L.A.col[e] == i) d = L.A.val[e];
      }
      xn[i] = x[i] + prm.omega * s / d;
    }
    std::copy(xn.begin(), xn.end(), x);
  }

  // pre-smoothing visits red then black, post-smoothing black then red
  void smooth(const AmgLevel& L, const double* f, double* x, bool pre) const {
    const int sweeps = pre ? prm.nu1 : prm.nu2;
    for (int s = 0; s < sweeps; ++s) {
      if (prm.smoother == 0) {
        gs_half(L, pre ? 0 : 1, f, x);
        gs_half(L, pre ? 1 : 0, f, x);
      } else {
        jacobi(L, f, x);
      }
    }
  }

  // x = V-cycle(level l) applied to f, starting from x = 0
  void vcycle(size_t l, const double* f, double* x) const {
    const AmgLevel& L = lv[l];
    if (l + 1 == lv.size()) {
      coarse.solve(f, x);
      return;
    }
    std::fill(x, x + L.A.n, 0.0);
    smooth(L, f, x, true);
    // restriction of the residual: f_c = P^T (f - A x)
    const AmgLevel& C = lv[l + 1];
    std::vector<double> fc(C.A.n, 0.0), xc(C.A.n, 0.0);
    for (int64_t i = 0; i < L.A.n; ++i) {
      double r = f[i];
      for (int32_t e = L.A.rowptr[i]; e < L.A.rowptr[i + 1]; ++e) r -= L.A.val[e] * x[L.A.col[e]];
      fc[L.agg[i]] += r;
    }
    vcycle(l + 1, fc.data(), xc.data());
    // prolongation with over-correction: x += s P x_c
    for (int64_t i = 0; i < L.A.n; ++i) x[i] += prm.overcorr * xc[L.agg[i]];
    smooth(L, f, x, false);
  }
};

// ---------------------------------------------------------------- preconditioners
struct Prec {
  virtual ~Prec() {}
  virtual void apply(const double* r, double* z) = 0;
};

struct IluPrec : Prec {
  Bsr A;                  // matrix in the factor ordering
  std::vector<double> lu;
  std::vector<int64_t> perm;  // perm[new] = old (empty: natural order)
  void apply(const double* r, double* z) override {
    const int bs = A.bs;
    if (perm.empty()) { ilu0_solve(A, lu, r, z); return; }
    std::vector<double> rp(A.n()), zp(A.n());
    for (int64_t i = 0; i < A.nb; ++i)
      for (int c = 0; c < bs; ++c) rp[i * bs + c] = r[perm[i] * bs + c];
    ilu0_solve(A, lu, rp.data(), zp.data());
    for (int64_t i = 0; i < A.nb; ++i)
      for (int c = 0; c < bs; ++c) z[perm[i] * bs + c] = zp[i * bs + c];
  }
};

// CPR-FPF (paper Alg. 2) on the decoupled matrix At = D_QI^{-1} A:
//   x = R^{-1} f;  r = f - At x;  x += Pi_p AMG(A_pp)^{-1} Pi_r r;
//   r = f - At x;  x += R^{-1} r
// with R = block ILU(0) of At and Pi_r / Pi_p taking / placing the pressure
// unknown (component 0) of each cell.  As a preconditioner of the original
// system it is applied to D_QI^{-1} v.
struct CprPrec : Prec {
  Bsr At;
  std::vector<double> w;  // per cell (g0, g1, g2): D_QI^{-1} row 0 = g0 e0 + g1 e1 + g2 e2
  IluPrec R;
  Amg amg;
  int stage = 0;  // 0 full CPR on D^{-1} v, 1 ILU only, 2 AMG only (Pi_p AMG Pi_r), 3 CPR on f as given
  // Learned coarse space (no counterpart in the paper): Z has one column
  // per tile holding the given pressure field zc on that tile's cells;
  // E = Z^T A~_pp Z with A~_pp the decoupled pressure block.  Every pressure
  // correction from the V-cycle gains Z E^{-1} Z^T fp.
  std::vector<double> zc;
  std::vector<int> tile;
  int ntiles = 0;
  DenseLU E;

  void coarse_correct(const double* fp, double* ep) const {
    if (ntiles == 0) return;
    std::vector<double> y(ntiles, 0.0), u(ntiles);
    for (size_t i = 0; i < zc.size(); ++i) y[tile[i]] += zc[i] * fp[i];
    E.solve(y.data(), u.data());
    for (size_t i = 0; i < zc.size(); ++i) ep[i] += zc[i] * u[tile[i]];
  }

  void cpr_decoupled(const double* f, double* x) {
    const int64_t n = At.n(), nb = At.nb;
    std::vector<double> r(n), Ax(n), fp(nb), ep(nb);
    R.apply(f, x);
    At.spmv(x, Ax.data());
    for (int64_t i = 0; i < n; ++i) r[i] = f[i] - Ax[i];
    for (int64_t i = 0; i < nb; ++i) fp[i] = r[3 * i];
    amg.vcycle(0, fp.data(), ep.data());
    coarse_correct(fp.data(), ep.data());
    for (int64_t i = 0; i < nb; ++i) x[3 * i] += ep[i];
    At.spmv(x, Ax.data());
    for (int64_t i = 0; i < n; ++i) r[i] = f[i] - Ax[i];
    std::vector<double> dx(n);
    R.apply(r.data(), dx.data());
    for (int64_t i = 0; i < n; ++i) x[i] += dx[i];
  }

  void apply(const double* v, double* z) override {
    const int64_t nb = At.nb;
    if (stage == 1) { R.apply(v, z); return; }
    if (stage == 2) {
      std::vector<double> fp(nb), ep(nb);
      for (int64_t i = 0; i < nb; ++i) fp[i] = v[3 * i];
      amg.vcycle(0, fp.data(), ep.data());
      coarse_correct(fp.data(), ep.data());
      for (int64_t i = 0; i < 3 * nb; ++i) z[i] = 0.0;
      for (int64_t i = 0; i < nb; ++i) z[3 * i] = ep[i];
      return;
    }
    if (stage == 3) { cpr_decoupled(v, z); return; }
    std::vector<double> f(v, v + 3 * nb);
    for (int64_t i = 0; i < nb; ++i) f[3 * i] = w[3 * i] * v[3 * i] + w[3 * i + 1] * v[3 * i + 1] + w[3 * i + 2] * v[3 * i + 2];
    cpr_decoupled(f.data(), z);
  }
};

// Quasi-IMPES decoupling (paper Sec. 3.2): D_QI = [[I, D_ps D_ss^{-1}, 0],
// [0, I, 0], [0, 0, I]] with D_ps = diag(A_ps), D_ss = diag(A_ss), read per
// cell on its own diagonal block: the pressure equation is the oil row 0,
// the saturation equations are rows 1 (water) and 2 (gas) against unknowns
// Sw (column 1) and Sg (column 2).  So D_QI^{-1} replaces row 0 of cell i by
// g . (row0, row1, row2) with g = (1, -a_01/a_11, -a_02/a_22) from A_ii.
// Where that leaves the cell's pressure pivot non-positive (injector cells
// flooded to residual oil, where the oil row carries no pressure
// information), the cell takes the exact local decoupling instead (the ABF
// alternative the paper names): g = row 0 of A_ii^{-1}, pivot 1.  g holds
// the three weights per cell.
int qi_decouple(const Bsr& A, Bsr& At, std::vector<double>& g) {
  At = A;
  g.assign(3 * A.nb, 0.0);
  for (int64_t i = 0; i < A.nb; ++i) {
    const double* D = nullptr;
    for (int32_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e)
      if (A.col[e] == i) D = &A.val[(size_t)e * 9];
    if (!D || D[4] == 0.0 || D[8] == 0.0) return kBreakdown;
    double gi[3] = {1.0, -D[1] / D[4], -D[2] / D[8]};
    const double pivot = gi[0] * D[0] + gi[1] * D[3] + gi[2] * D[6];
    if (!(pivot > 0.0)) {
      // row 0 of A_ii^{-1}: solve A_ii^T y = e_0
      double Dt[9], e0[3] = {1.0, 0.0, 0.0};
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Dt[3 * r + c] = D[3 * c + r];
      if (!block_solve(3, Dt, e0, gi)) return kBreakdown;
    }
    g[3 * i] = gi[0];
    g[3 * i + 1] = gi[1];
    g[3 * i + 2] = gi[2];
    const double Dinv[9] = {gi[0], gi[1], gi[2], 0.0, 1.0, 0.0, 0.0, 0.0, 1.0};
    for (int32_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e)
      block_mul(3, Dinv, &A.val[(size_t)e * 9], &At.val[(size_t)e * 9]);
  }
  return kOk;
}

// A_pp: the (0, 0) entry of every block, on the block pattern
Csr pressure_block(const Bsr& A) {
  Csr C;
  C.n = A.nb;
  C.rowptr = A.rowptr;
  C.col = A.col;
  C.val.resize(A.col.size());
  for (size_t e = 0; e < A.col.size(); ++e) C.val[e] = A.val[e * 9];
  return C;
}

// Red-black order of a structured grid: cells with (i + j + k) even first,
// each colour in natural order.  perm[new] = old.
std::vector<int64_t> red_black_perm(int nx, int ny, int nz) {
  std::vector<int64_t> perm;
  const int64_t N = (int64_t)nx * ny * nz;
  perm.reserve(N);
  for (int col = 0; col < 2; ++col)
    for (int64_t c = 0; c < N; ++c) {
      const int64_t i = c % nx, j = (c / nx) % ny, k = c / ((int64_t)nx * ny);
      if (((i + j + k) & 1) == col) perm.push_back(c);
    }
  return perm;
}

// Neumaier-compensated accumulator
struct KSum {
  double s = 0, c = 0;
  void add(double x) {
    const double t = s + x;
    if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

}  // namespace

// ====================================================================== C ABI
extern "C" {

void or_bsr_spmv(int64_t nb, int bs, const int32_t* rowptr, const int32_t* col, const double* val,
                 const double* x, double* y) {
  Bsr A = make_bsr(nb, bs, rowptr, col, val);
  A.spmv(x, y);
}

// y = A x with the block rows split into T contiguous ranges, one host
// thread each (no copy of A: the benchmark times this as the CPU's SpMV
// bandwidth).  Same arithmetic as or_bsr_spmv row by row.
void or_bsr_spmv_threads(int64_t nb, int bs, const int32_t* rowptr, const int32_t* col, const double* val,
                         const double* x, double* y, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  auto rows = [=](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i)
      for (int r = 0; r < bs; ++r) {
        double acc = 0.0;
        for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
          const double* blk = val + (size_t)e * bs * bs + bs * r;
          const double* xc = x + (size_t)col[e] * bs;
          for (int c = 0; c < bs; ++c) acc += blk[c] * xc[c];
        }
        y[i * bs + r] = acc;
      }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t) {
    const int64_t i0 = nb * t / nthreads, i1 = nb * (t + 1) / nthreads;
    pool.emplace_back(rows, i0, i1);
  }
  for (auto& th : pool) th.join();
}

// out = D_QI^{-1} A (same pattern), g[3 nb] = the row-0 weights of D_QI^{-1} per cell
int or_qi_decouple(int64_t nb, const int32_t* rowptr, const int32_t* col, const double* val,
                   double* out, double* w) {
  Bsr A = make_bsr(nb, 3, rowptr, col, val), At;
  std::vector<double> ww;
  int rc = qi_decouple(A, At, ww);
  if (rc != kOk) return rc;
  std::copy(At.val.begin(), At.val.end(), out);
  std::copy(ww.begin(), ww.end(), w);
  return kOk;
}

// B = P A P^T, perm[new] = old; out arrays sized like A's
void or_bsr_permute(int64_t nb, int bs, const int32_t* rowptr, const int32_t* col, const double* val,
                    const int64_t* perm, int32_t* orow, int32_t* ocol, double* oval) {
  Bsr A = make_bsr(nb, bs, rowptr, col, val);
  Bsr B = permute(A, perm);
  std::copy(B.rowptr.begin(), B.rowptr.end(), orow);
  std::copy(B.col.begin(), B.col.end(), ocol);
  std::copy(B.val.begin(), B.val.end(), oval);
}

int or_bsr_ilu0(int64_t nb, int bs, const int32_t* rowptr, const int32_t* col, const double* val, double* lu) {
  Bsr A = make_bsr(nb, bs, rowptr, col, val);
  std::vector<double> f;
  int rc = ilu0_factor(A, f);
  if (rc == kOk) std::copy(f.begin(), f.end(), lu);
  return rc;
}

void or_bsr_ilu0_solve(int64_t nb, int bs, const int32_t* rowptr, const int32_t* col, const double* lu,
                       const double* r, double* z) {
  Bsr A = make_bsr(nb, bs, rowptr, col, lu);
  ilu0_solve(A, A.val, r, z);
}

int or_dense_solve(int n, const double* A, const double* b, double* x) {
  DenseLU lu;
  int rc = lu.factor(n, A);
  if (rc != kOk) return rc;
  lu.solve(b, x);
  return kOk;
}

void or_red_black_perm(int nx, int ny, int nz, int64_t* perm) {
  auto p = red_black_perm(nx, ny, nz);
  std::copy(p.begin(), p.end(), perm);
}

// ---- AMG on a scalar CSR matrix living on an nx x ny x nz grid
void* or_amg_create(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                    int nx, int ny, int nz, int smoother, int nu1, int nu2, double omega,
                    double overcorr, int coarse_max, int max_levels, int* status) {
  Csr A;
  A.n = n;
  A.rowptr.assign(rowptr, rowptr + n + 1);
  A.col.assign(col, col + rowptr[n]);
  A.val.assign(val, val + rowptr[n]);
  AmgParams p;
  p.smoother = smoother; p.nu1 = nu1; p.nu2 = nu2; p.omega = omega;
  p.overcorr = overcorr; p.coarse_max = coarse_max; p.max_levels = max_levels;
  auto* amg = new Amg();
  *status = amg->setup(A, nx, ny, nz, p);
  return amg;
}
int or_amg_nlevels(void* h) { return (int)static_cast<Amg*>(h)->lv.size(); }
void or_amg_level_dims(void* h, int l, int* dims) {
  const AmgLevel& L = static_cast<Amg*>(h)->lv[l];
  dims[0] = L.nx; dims[1] = L.ny; dims[2] = L.nz;
}
// copy of level l's matrix: returns nnz; arrays may be NULL to query
int64_t or_amg_level_matrix(void* h, int l, int32_t* rowptr, int32_t* col, double* val) {
  const Csr& A = static_cast<Amg*>(h)->lv[l].A;
  if (rowptr) std::copy(A.rowptr.begin(), A.rowptr.end(), rowptr);
  if (col) std::copy(A.col.begin(), A.col.end(), col);
  if (val) std::copy(A.val.begin(), A.val.end(), val);
  return (int64_t)A.col.size();
}
void or_amg_vcycle(void* h, const double* f, double* x) { static_cast<Amg*>(h)->vcycle(0, f, x); }
void or_amg_destroy(void* h) { delete static_cast<Amg*>(h); }

// ---- preconditioner handles for GMRES
// ILU(0) of A in natural order (ordering 0) or red-black order of the grid (1)
void* or_prec_ilu0_create(int64_t nb, int bs, const int32_t* rowptr, const int32_t* col, const double* val,
                          int ordering, int nx, int ny, int nz, int* status) {
  auto* p = new IluPrec();
  Bsr A = make_bsr(nb, bs, rowptr, col, val);
  if (ordering == 1) {
    p->perm = red_black_perm(nx, ny, nz);
    p->A = permute(A, p->perm.data());
  } else {
    p->A = A;
  }
  *status = ilu0_factor(p->A, p->lu);
  return p;
}

// CPR-FPF of the (undecoupled) 3x3 BSR matrix A on an nx x ny x nz grid.
// ILU(0) ordering: 0 natural, 1 red-black.  stage: 0 full preconditioner
// z = CPR(D_QI^{-1} v); 1 R^{-1} only; 2 Pi_p AMG^{-1} Pi_r only; 3 CPR on
// an already decoupled input.
void* or_prec_cpr_create(int64_t nb, const int32_t* rowptr, const int32_t* col, const double* val,
                         int nx, int ny, int nz, int ordering,
                         int smoother, int nu1, int nu2, double omega, double overcorr,
                         int coarse_max, int max_levels, int stage, int* status) {
  auto* p = new CprPrec();
  Bsr A = make_bsr(nb, 3, rowptr, col, val);
  p->stage = stage;
  *status = qi_decouple(A, p->At, p->w);
  if (*status != kOk) return p;
  if (ordering == 1) {
    p->R.perm = red_black_perm(nx, ny, nz);
    p->R.A = permute(p->At, p->R.perm.data());
  } else {
    p->R.A = p->At;
  }
  *status = ilu0_factor(p->R.A, p->R.lu);
  if (*status != kOk) return p;
  AmgParams ap;
  ap.smoother = smoother; ap.nu1 = nu1; ap.nu2 = nu2; ap.omega = omega;
  ap.overcorr = overcorr; ap.coarse_max = coarse_max; ap.max_levels = max_levels;
  *status = p->amg.setup(pressure_block(p->At), nx, ny, nz, ap);
  return p;
}

// Learned coarse space of a CPR preconditioner from or_prec_cpr_create:
// zc (one value per cell, natural order) restricted to tiles of tx x ty x tz
// cells; tile t = a + ntx (b + nty c) for the tile at (a, b, c).  A tile
// where zc vanishes gets E_tt = 1 (its column of Z is zero).  zc = NULL
// removes the space.  Returns 0, or -5 if E is singular.
int or_prec_cpr_set_coarse(void* h, const double* zc, int nx, int ny, int nz, int tx, int ty, int tz) {
  auto* p = static_cast<CprPrec*>(h);
  p->ntiles = 0;
  p->zc.clear();
  p->tile.clear();
  if (!zc) return kOk;
  const int ntx = (nx + tx - 1) / tx, nty = (ny + ty - 1) / ty, ntz = (nz + tz - 1) / tz;
  const int nt = ntx * nty * ntz;
  const int64_t n = (int64_t)nx * ny * nz;
  std::vector<int> tile(n);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) tile[i + (int64_t)nx * (j + (int64_t)ny * k)] = i / tx + ntx * (j / ty + nty * (k / tz));
  // E[s][t] = sum over cells c in s and pressure couplings (c, d) with d in t of zc_c A~_pp[c][d] zc_d
  const Csr App = pressure_block(p->At);
  std::vector<double> E((size_t)nt * nt, 0.0), zz(nt, 0.0);
  for (int64_t c = 0; c < n; ++c) {
    zz[tile[c]] += zc[c] * zc[c];
    for (int32_t e = App.rowptr[c]; e < App.rowptr[c + 1]; ++e)
      E[(size_t)tile[c] * nt + tile[App.col[e]]] += zc[c] * App.val[e] * zc[App.col[e]];
  }
  for (int t = 0; t < nt; ++t)
    if (zz[t] == 0.0) E[(size_t)t * nt + t] = 1.0;
  if (p->E.factor(nt, E.data()) != kOk) return kBreakdown;
  p->zc.assign(zc, zc + n);
  p->tile = tile;
  p->ntiles = nt;
  return kOk;
}

// The coarse correction alone: ep = Z E^{-1} Z^T fp (natural order)
void or_prec_cpr_coarse_apply(void* h, const double* fp, double* ep) {
  auto* p = static_cast<CprPrec*>(h);
  for (size_t i = 0; i < p->zc.size(); ++i) ep[i] = 0.0;
  p->coarse_correct(fp, ep);
}

void or_prec_apply(void* h, const double* r, double* z) { static_cast<Prec*>(h)->apply(r, z); }
void or_prec_destroy(void* h) { delete static_cast<Prec*>(h); }

// ||b - A x||_2 / ||b||_2 with compensated sums (||b - A x|| if b = 0)
double or_rel_residual(int64_t nb, int bs, const int32_t* rowptr, const int32_t* col, const double* val,
                       const double* b, const double* x) {
  KSum rr, bb;
  for (int64_t i = 0; i < nb; ++i)
    for (int r = 0; r < bs; ++r) {
      KSum s;
      s.add(b[i * bs + r]);
      for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
        for (int c = 0; c < bs; ++c) s.add(-val[(size_t)e * bs * bs + bs * r + c] * x[(size_t)col[e] * bs + c]);
      const double ri = s.value();
      rr.add(ri * ri);
      bb.add(b[i * bs + r] * b[i * bs + r]);
    }
  const double nb2 = bb.value();
  return nb2 > 0 ? std::sqrt(rr.value() / nb2) : std::sqrt(rr.value());
}

// Restarted GMRES(m), right preconditioned by `prec` (NULL: none), modified
// Gram-Schmidt and Givens rotations.  Iterates until ||b - A x|| <= tol ||b||
// holds for the recomputed residual or `maxit` iterations were spent.
// x holds the initial guess on entry.  info = {iterations, true relative
// residual, restarts}.  Returns 0, or -7 when maxit was reached first.
int or_gmres(int64_t nb, int bs, const int32_t* rowptr, const int32_t* col, const double* val,
             const double* b, double* x, int m, int maxit, double tol, void* prec, double* info) {
  Bsr A = make_bsr(nb, bs, rowptr, col, val);
  Prec* P = static_cast<Prec*>(prec);
  const int64_t n = A.n();
  std::vector<double> r(n), w(n);
  std::vector<std::vector<double>> V(m + 1, std::vector<double>(n)), Z(m, std::vector<double>(n));
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  const double bnorm = std::sqrt(dot(n, b, b));
  const double target = tol * (bnorm > 0 ? bnorm : 1.0);
  int its = 0, restarts = 0;
  double relres = 0;
  auto true_residual = [&]() {
    A.spmv(x, w.data());
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - w[i];
    return std::sqrt(dot(n, r.data(), r.data()));
  };
  double beta = true_residual();
  while (true) {
    relres = beta / (bnorm > 0 ? bnorm : 1.0);
    if (beta <= target || its >= maxit) break;
    for (int64_t i = 0; i < n; ++i) V[0][i] = r[i] / beta;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m && its < maxit; ++j) {
      if (P) P->apply(V[j].data(), Z[j].data());
      else std::copy(V[j].begin(), V[j].end(), Z[j].begin());
      A.spmv(Z[j].data(), w.data());
      const double wnorm0 = std::sqrt(dot(n, w.data(), w.data()));
      for (int i = 0; i <= j; ++i) {
        const double h = dot(n, w.data(), V[i].data());
        H[(size_t)i * m + j] = h;
        for (int64_t t = 0; t < n; ++t) w[t] -= h * V[i][t];
      }
      const double hn = std::sqrt(dot(n, w.data(), w.data()));
      H[(size_t)(j + 1) * m + j] = hn;
      const bool happy = hn <= 1e-14 * wnorm0;
      if (!happy)
        for (int64_t t = 0; t < n; ++t) V[j + 1][t] = w[t] / hn;
      for (int i = 0; i < j; ++i) {  // previous rotations
        const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
      const double d = std::hypot(a, c);
      cs[j] = a / d;
      sn[j] = c / d;
      H[(size_t)j * m + j] = d;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      k = j + 1;
      if (std::fabs(g[j + 1]) <= target || happy) break;
    }
    for (int i = k - 1; i >= 0; --i) {  // H y = g
      double s = g[i];
      for (int t = i + 1; t < k; ++t) s -= H[(size_t)i * m + t] * y[t];
      y[i] = s / H[(size_t)i * m + i];
    }
    for (int i = 0; i < k; ++i)
      for (int64_t t = 0; t < n; ++t) x[t] += y[i] * Z[i][t];
    beta = true_residual();
    ++restarts;
  }
  info[0] = its;
  info[1] = relres;
  info[2] = restarts;
  return beta <= target ? kOk : kNotConverged;
}

// Right-preconditioned BiCGSTAB (van der Vorst, SIAM J. Sci. Stat. Comput.
// 13, 1992), preconditioner `prec` (NULL: none).  Each iteration applies the
// preconditioner twice and A twice: the BiCG step p -> v = A M^{-1} p with
// alpha = rho / (rt, v), then the minimal-residual step s -> t = A M^{-1} s
// with omega = (t, s) / (t, t).  When the recursive residual meets
// tol ||b|| the true residual b - A x is recomputed; if it does not meet the
// tolerance, or a scalar of the recurrence vanishes, the iteration restarts
// from the true residual with a new shadow vector rt = r.  x holds the
// initial guess on entry.  info = {iterations, true relative residual,
// restarts}.  Returns 0, -7 when maxit was reached first, -6 on a breakdown
// right after a restart.
int or_bicgstab(int64_t nb, int bs, const int32_t* rowptr, const int32_t* col, const double* val,
                const double* b, double* x, int maxit, double tol, void* prec, double* info) {
  Bsr A = make_bsr(nb, bs, rowptr, col, val);
  Prec* P = static_cast<Prec*>(prec);
  const int64_t n = A.n();
  std::vector<double> r(n), rt(n), p(n), v(n), s(n), t(n), ph(n), sh(n);
  const double bnorm = std::sqrt(dot(n, b, b));
  const double target = tol * (bnorm > 0 ? bnorm : 1.0);
  auto apply_prec = [&](const double* in, double* out) {
    if (P) P->apply(in, out);
    else std::copy(in, in + n, out);
  };
  auto true_residual = [&]() {
    A.spmv(x, v.data());
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - v[i];
    return std::sqrt(dot(n, r.data(), r.data()));
  };
  int its = 0, restarts = 0, status = kNotConverged;
  double rnorm = true_residual();
  bool fresh = true;  // no iteration since the last (re)start
  while (rnorm > target && its < maxit) {
    // (re)start: shadow vector rt = r, p = v = 0, rho_prev = alpha = omega = 1
    rt = r;
    std::fill(p.begin(), p.end(), 0.0);
    std::fill(v.begin(), v.end(), 0.0);
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    bool restart = false;
    while (!restart && its < maxit) {
      const double rho = dot(n, rt.data(), r.data());
      if (rho == 0.0) { restart = true; break; }
      const double beta = (rho / rho_prev) * (alpha / omega);
      for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
      apply_prec(p.data(), ph.data());
      A.spmv(ph.data(), v.data());
      const double rtv = dot(n, rt.data(), v.data());
      if (rtv == 0.0) { restart = true; break; }
      alpha = rho / rtv;
      for (int64_t i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
      ++its;
      fresh = false;
      if (std::sqrt(dot(n, s.data(), s.data())) <= target) {
        for (int64_t i = 0; i < n; ++i) x[i] += alpha * ph[i];
        restart = true;  // recompute the true residual below
        break;
      }
      apply_prec(s.data(), sh.data());
      A.spmv(sh.data(), t.data());
      const double tt = dot(n, t.data(), t.data());
      if (tt == 0.0) {
        for (int64_t i = 0; i < n; ++i) x[i] += alpha * ph[i];
        restart = true;
        break;
      }
      omega = dot(n, t.data(), s.data()) / tt;
      for (int64_t i = 0; i < n; ++i) {
        x[i] += alpha * ph[i] + omega * sh[i];
        r[i] = s[i] - omega * t[i];
      }
      rho_prev = rho;
      if (omega == 0.0 || std::sqrt(dot(n, r.data(), r.data())) <= target) restart = true;
    }
    const double prev = rnorm;
    rnorm = true_residual();
    ++restarts;
    if (rnorm <= target) break;
    if (fresh && rnorm >= prev) {  // broke down before any progress
      status = kBreakdown;
      break;
    }
    fresh = true;
  }
  if (rnorm <= target) status = kOk;
  info[0] = its;
  info[1] = rnorm / (bnorm > 0 ? bnorm : 1.0);
  info[2] = restarts;
  return status;
}

}  // extern "C"
