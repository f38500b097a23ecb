// Black-oil residual and Jacobian assembly: the seeded input generator of the
// linear solver.  It produces the Newton system A dx = b of one step of the
// fully implicit three-phase black-oil model, which is the input both the GPU
// solver and the CPU oracle consume.  It holds none of the solver's
// arithmetic (no SpMV, decoupling, ILU, AMG or Krylov code).
//
// What it computes (paper Sec. 2.1, Eq. 3 with its closure relations, the
// no-flow boundary, Stone II relative permeability; Sec. 2.3 Eq. 4 Peaceman
// wells under fixed bottom-hole pressure; Sec. 3.1 Alg. 1 Newton convention):
//
//   R_c,i = V_i/(5.615 dt) [M_c(x_i) - M_c(x_i^n)]
//           - sum_{j in nb(i)} T_ij sum_alpha (x_c,alpha lambda_alpha)_up dPhi_alpha,ij
//           - Q_c,i
//   b = -R(x),  A = dR/dx  (exact forward-mode derivatives, not differences)
//
// Unknowns per cell: (p, Sw, Sg) = (oil pressure, water and gas saturation).
// Equations per cell: (oil, water, gas) components.  Field units: ft, psi,
// mD, cp, day, stb, Mscf.  Cell c = i + nx (j + ny k); depth grows with k.
//
// Block layout of the output: BSR with 3x3 blocks, row-major inside a block
// (row = equation, column = unknown), columns of a block row sorted
// ascending, every 7-point neighbour present (also where its value is zero).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

namespace {

// ---------------------------------------------------------------- dual numbers
template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0) { for (int i = 0; i < N; ++i) d[i] = 0; }
  Dual(double a) : v(a) { for (int i = 0; i < N; ++i) d[i] = 0; }
  static Dual var(double a, int slot) { Dual r(a); r.d[slot] = 1.0; return r; }
};
template <int N> Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) { Dual<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int N> Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) { Dual<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int N> Dual<N> operator-(const Dual<N>& a) { Dual<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r; }
template <int N> Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) { Dual<N> r; r.v = a.v * b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int N> Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) { Dual<N> r; r.v = a.v / b.v; for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v); return r; }
template <int N> Dual<N> operator+(const Dual<N>& a, double b) { Dual<N> r = a; r.v += b; return r; }
template <int N> Dual<N> operator+(double b, const Dual<N>& a) { return a + b; }
template <int N> Dual<N> operator-(const Dual<N>& a, double b) { Dual<N> r = a; r.v -= b; return r; }
template <int N> Dual<N> operator-(double b, const Dual<N>& a) { return (-a) + b; }
template <int N> Dual<N> operator*(const Dual<N>& a, double b) { Dual<N> r; r.v = a.v * b; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b; return r; }
template <int N> Dual<N> operator*(double b, const Dual<N>& a) { return a * b; }
template <int N> Dual<N> operator/(const Dual<N>& a, double b) { return a * (1.0 / b); }
template <int N> Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> Dual<N> dmax0(const Dual<N>& a) { return a.v > 0 ? a : Dual<N>(0.0); }
template <int N> Dual<N> sq(const Dual<N>& a) { return a * a; }

// Lift a cell-local dual (3 derivative slots) into a face dual (6 slots);
// `off` = 0 for the first cell of the face, 3 for the second.
Dual<6> lift(const Dual<3>& a, int off) {
  Dual<6> r(a.v);
  for (int i = 0; i < 3; ++i) r.d[off + i] = a.d[i];
  return r;
}

}  // namespace

extern "C" {

// Fluid, rock and saturation-function constants.  The paper fixes none for
// synthetic cases; the defaults the Python side fills in are the readings
// documented with the generator.
typedef struct {
  double pref;                     // psi, reference pressure of the linear tables
  double bw0, cw, muw;             // Bw = bw0 (1 - cw (p - pref)); water viscosity (cp)
  double bo0, dbo, rs0, drs, muo;  // Bo = bo0 + dbo (p - pref); Rs (Mscf/stb) = rs0 + drs (p - pref)
  double bg0, dbg, mug;            // Bg (rb/Mscf) = bg0 - dbg (p - pref)
  double rhow_sc, rhoo_sc, rhog_sc;// stock-tank densities, lb/ft^3
  double cr;                       // rock compressibility, 1/psi: phi = phi0 (1 + cr (p - pref))
  double swc, sorw, sorg, sgc;     // saturation end points
  double nw, now, ng, nog;         // Corey exponents
  double gravity;                  // 1 = hydrostatic terms on, 0 = off
} bg_fluid;

typedef struct {
  int32_t nx, ny, nz;
  double dx, dy, dz;
} bg_grid;

// Test-only Dirichlet pressure on the x = 0 and x = L faces (a half-cell
// boundary transmissibility; the boundary fluid has the adjacent cell's
// saturations).  enabled = 0 keeps the paper's no-flow boundary.
typedef struct {
  int32_t enabled;
  double p_left, p_right;
} bg_bc;

}  // extern "C"

namespace {

constexpr double kDarcy = 0.001127;  // bbl cp / (day ft^2 psi mD)
constexpr double kBblFt3 = 5.615;    // ft^3 per bbl

struct Props {  // everything a cell contributes, as functions of its unknowns
  Dual<3> phi, bw, bo, bg, rs;
  Dual<3> lw, lo, lg;        // mobilities k_r / (mu B)
  Dual<3> lt_res_w;          // total reservoir mobility / Bw (water injector)
  Dual<3> gw, go, gg;        // phase gravity gradients rho / 144, psi/ft
  Dual<3> mw, mo, mg;        // component masses per pore... per bulk volume
};

// Two-phase Corey curves and Stone II three-phase oil relative permeability
// (paper Sec. 2.1: K_ro from the Stone II formula).
template <int N>
void relperm(const bg_fluid& f, const Dual<N>& sw, const Dual<N>& sg,
             Dual<N>& krw, Dual<N>& kro, Dual<N>& krg) {
  const double dw = 1.0 - f.swc - f.sorw;
  const double dg = 1.0 - f.swc - f.sorg - f.sgc;
  Dual<N> swn = dmax0((sw - f.swc) / dw);
  Dual<N> sown = dmax0((1.0 - sw - f.sorw) / dw);
  Dual<N> sgn = dmax0((sg - f.sgc) / dg);
  Dual<N> sogn = dmax0((1.0 - sg - f.swc - f.sorg) / dg);
  krw = Dual<N>(1.0); krg = Dual<N>(1.0);
  Dual<N> krow(1.0), krog(1.0);
  // integer Corey exponents are the common case; general exponents via pow
  auto cpow = [](const Dual<N>& s, double e) {
    if (e == 2.0) return s * s;
    Dual<N> r(std::pow(s.v, e));
    double dv = s.v > 0 ? e * std::pow(s.v, e - 1.0) : 0.0;
    for (int i = 0; i < N; ++i) r.d[i] = dv * s.d[i];
    return r;
  };
  krw = cpow(swn, f.nw);
  krow = cpow(sown, f.now);
  krg = cpow(sgn, f.ng);
  krog = cpow(sogn, f.nog);
  // k_rocw = k_row at connate water
  const double krocw = std::pow(std::max(0.0, (1.0 - f.swc - f.sorw) / dw), f.now);
  kro = dmax0(krocw * ((krow / krocw + krw) * (krog / krocw + krg) - krw - krg));
}

Props cell_props(const bg_fluid& f, double phi0, double p_, double sw_, double sg_) {
  Props c;
  Dual<3> p = Dual<3>::var(p_, 0), sw = Dual<3>::var(sw_, 1), sg = Dual<3>::var(sg_, 2);
  Dual<3> so = 1.0 - sw - sg;
  Dual<3> dp = p - f.pref;
  c.phi = phi0 * (1.0 + f.cr * dp);
  c.bw = f.bw0 * (1.0 - f.cw * dp);
  c.bo = f.bo0 + f.dbo * dp;
  c.rs = f.rs0 + f.drs * dp;
  c.bg = f.bg0 - f.dbg * dp;
  Dual<3> krw, kro, krg;
  relperm(f, sw, sg, krw, kro, krg);
  c.lw = krw / (f.muw * c.bw);
  c.lo = kro / (f.muo * c.bo);
  c.lg = krg / (f.mug * c.bg);
  c.lt_res_w = (krw / f.muw + kro / f.muo + krg / f.mug) / c.bw;
  // reservoir phase densities (lb/ft^3) -> gradients (psi/ft)
  Dual<3> rhow = f.rhow_sc / c.bw;
  Dual<3> rhoo = (f.rhoo_sc * kBblFt3 + c.rs * (1000.0 * f.rhog_sc)) / (kBblFt3 * c.bo);
  Dual<3> rhog = (1000.0 * f.rhog_sc) / (kBblFt3 * c.bg);
  c.gw = f.gravity * rhow / 144.0;
  c.go = f.gravity * rhoo / 144.0;
  c.gg = f.gravity * rhog / 144.0;
  // component amounts per unit pore... per unit bulk volume (stb or Mscf per rb)
  c.mw = c.phi * sw / c.bw;
  c.mo = c.phi * so / c.bo;
  c.mg = c.phi * (sg / c.bg + c.rs * so / c.bo);
  return c;
}

double cell_mass_value(const bg_fluid& f, double phi0, double p, double sw, double sg, int comp) {
  Props c = cell_props(f, phi0, p, sw, sg);
  return comp == 0 ? c.mo.v : comp == 1 ? c.mw.v : c.mg.v;
}

struct Assembler {
  const bg_grid& g;
  const bg_fluid& f;
  int64_t N;
  const int32_t* rowptr;
  const int32_t* col;
  double* R;
  double* val;
  // add a 3x3 derivative block (equation rows x unknown columns) to A[row][colcell]
  void add_block(int64_t row, int64_t colcell, const double blk[3][3]) {
    if (!val) return;
    for (int32_t e = rowptr[row]; e < rowptr[row + 1]; ++e) {
      if (col[e] == colcell) {
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) val[9 * (int64_t)e + 3 * r + c] += blk[r][c];
        return;
      }
    }
  }
};


// Flux into node a from node b through a connection of transmissibility T,
// computed once and added with opposite signs to both nodes' residuals and
// Jacobian rows.  za, zb: depths of the two nodes.
void add_face(Assembler& as, const std::vector<Props>& P, const double* x, double za, double zb, int64_t a,
              int64_t b, double T, double* R) {
  const Props& A = P[a];
  const Props& B = P[b];
  Dual<6> pa = Dual<6>::var(x[3 * a], 0), pb = Dual<6>::var(x[3 * b], 3);
  const double dz = zb - za;
  // phase potential differences Phi_b - Phi_a, face density = mean of the two nodes
  Dual<6> dphi_o = (pb - pa) - 0.5 * (lift(A.go, 0) + lift(B.go, 3)) * dz;
  Dual<6> dphi_w = (pb - pa) - 0.5 * (lift(A.gw, 0) + lift(B.gw, 3)) * dz;
  Dual<6> dphi_g = (pb - pa) - 0.5 * (lift(A.gg, 0) + lift(B.gg, 3)) * dz;
  // upstream node: b if the potential of b is higher; on a tie the lower index
  auto up = [&](const Dual<6>& d, const Dual<3>& qa, const Dual<3>& qb) {
    if (d.v > 0) return lift(qb, 3);
    if (d.v < 0) return lift(qa, 0);
    return a < b ? lift(qa, 0) : lift(qb, 3);
  };
  Dual<6> fo = T * up(dphi_o, A.lo, B.lo) * dphi_o;
  Dual<6> fw = T * up(dphi_w, A.lw, B.lw) * dphi_w;
  Dual<6> fg = T * (up(dphi_o, A.rs * A.lo, B.rs * B.lo) * dphi_o + up(dphi_g, A.lg, B.lg) * dphi_g);
  const Dual<6>* F[3] = {&fo, &fw, &fg};
  double ba[3][3], bb[3][3];
  for (int comp = 0; comp < 3; ++comp) {
    R[3 * a + comp] -= F[comp]->v;
    R[3 * b + comp] += F[comp]->v;
    for (int u = 0; u < 3; ++u) { ba[comp][u] = F[comp]->d[u]; bb[comp][u] = F[comp]->d[3 + u]; }
  }
  double m[3][3];
  for (int r = 0; r < 3; ++r) for (int u = 0; u < 3; ++u) m[r][u] = -ba[r][u];
  as.add_block(a, a, m);
  for (int r = 0; r < 3; ++r) for (int u = 0; u < 3; ++u) m[r][u] = -bb[r][u];
  as.add_block(a, b, m);
  as.add_block(b, a, ba);
  as.add_block(b, b, bb);
}

// accumulation of node c: V / (5.615 dt) (M(x) - M(x_n))
void add_accumulation(Assembler& as, const bg_fluid& f, const Props& Pc, double phi0, const double* xn_c, double V,
                      double dt, int64_t c, double* R) {
  const double s = V / (kBblFt3 * dt);
  const Dual<3>* m[3] = {&Pc.mo, &Pc.mw, &Pc.mg};
  double blk[3][3];
  for (int comp = 0; comp < 3; ++comp) {
    const double mn = cell_mass_value(f, phi0, xn_c[0], xn_c[1], xn_c[2], comp);
    R[3 * c + comp] += s * (m[comp]->v - mn);
    for (int u = 0; u < 3; ++u) blk[comp][u] = s * m[comp]->d[u];
  }
  as.add_block(c, c, blk);
}

// wells under fixed bottom-hole pressure (paper Eq. 4) on the perforated nodes:
// the rate into node c is WI * mobility * (p_h - p - rho g (z_h - z))
void add_wells(Assembler& as, const std::vector<Props>& P, const double* x, const double* depth, int32_t nw,
               const int32_t* wtype, const double* bhp, const double* dref, const int32_t* perf_ptr,
               const int32_t* perf_cells, const double* perf_wi, double* R) {
  for (int32_t w = 0; w < nw; ++w) {
    for (int32_t e = perf_ptr[w]; e < perf_ptr[w + 1]; ++e) {
      const int64_t c = perf_cells[e];
      const Props& C = P[c];
      const double WI = perf_wi[e];
      Dual<3> p = Dual<3>::var(x[3 * c], 0);
      const double dzh = dref[w] - depth[c];
      Dual<3> dpo = bhp[w] - p - C.go * dzh;
      Dual<3> dpw = bhp[w] - p - C.gw * dzh;
      Dual<3> dpg = bhp[w] - p - C.gg * dzh;
      Dual<3> qo(0.0), qw(0.0), qg(0.0);
      if (wtype[w] == 0) {
        qw = WI * C.lt_res_w * dpw;  // water injector: total mobility
      } else {
        qo = WI * C.lo * dpo;
        qw = WI * C.lw * dpw;
        qg = WI * (C.rs * C.lo * dpo + C.lg * dpg);
      }
      const Dual<3>* Q[3] = {&qo, &qw, &qg};
      double blk[3][3];
      for (int comp = 0; comp < 3; ++comp) {
        R[3 * c + comp] -= Q[comp]->v;
        for (int u = 0; u < 3; ++u) blk[comp][u] = -Q[comp]->d[u];
      }
      as.add_block(c, c, blk);
    }
  }
}

}  // namespace

extern "C" {

// Peaceman well index for a vertical well in a cell of size dx x dy x dz with
// permeabilities kx, ky (mD): WI = 0.001127 2 pi sqrt(kx ky) dz / (ln(ro/rw) + skin),
// ro from Peaceman's anisotropic equivalent radius (paper Sec. 2.3, Eq. 4 and
// the Peaceman reference it cites).
double bg_peaceman_wi(double kx, double ky, double dx, double dy, double dz, double rw, double skin) {
  const double a = std::sqrt(ky / kx), b = std::sqrt(kx / ky);
  const double ro = 0.28 * std::sqrt(a * dx * dx + b * dy * dy) / (std::pow(ky / kx, 0.25) + std::pow(kx / ky, 0.25));
  return kDarcy * 2.0 * M_PI * std::sqrt(kx * ky) * dz / (std::log(ro / rw) + skin);
}

// Relative permeabilities at one saturation pair: out = {krw, kro, krg}.
void bg_relperm(const bg_fluid* f, double sw, double sg, double* out) {
  Dual<1> w(sw), g(sg), krw, kro, krg;
  relperm(*f, w, g, krw, kro, krg);
  out[0] = krw.v; out[1] = kro.v; out[2] = krg.v;
}

// Component amount per unit bulk volume of a cell: comp 0 oil (stb/rb),
// 1 water (stb/rb), 2 gas (Mscf/rb).
double bg_cell_mass(const bg_fluid* f, double phi0, double p, double sw, double sg, int comp) {
  return cell_mass_value(*f, phi0, p, sw, sg, comp);
}

// Number of 3x3 blocks of the 7-point pattern.
int64_t bg_nnzb(const bg_grid* g) {
  const int64_t nx = g->nx, ny = g->ny, nz = g->nz;
  return nx * ny * nz + 2 * ((nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1));
}

// Fill the BSR pattern (rowptr[N+1], col[nnzb]) of the 7-point stencil.
void bg_pattern(const bg_grid* g, int32_t* rowptr, int32_t* col) {
  const int64_t nx = g->nx, ny = g->ny, nz = g->nz;
  int64_t e = 0;
  rowptr[0] = 0;
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        const int64_t c = i + nx * (j + ny * k);
        if (k > 0) col[e++] = (int32_t)(c - nx * ny);
        if (j > 0) col[e++] = (int32_t)(c - nx);
        if (i > 0) col[e++] = (int32_t)(c - 1);
        col[e++] = (int32_t)c;
        if (i < nx - 1) col[e++] = (int32_t)(c + 1);
        if (j < ny - 1) col[e++] = (int32_t)(c + nx);
        if (k < nz - 1) col[e++] = (int32_t)(c + nx * ny);
        rowptr[c + 1] = (int32_t)e;
      }
}

// Assemble R(x) (3N, component order oil, water, gas) and, if val != NULL,
// the Jacobian values val[9 nnzb] on the pattern from bg_pattern.
//   kx, ky, kz, phi0, depth: per cell.  x, xn: current and previous state (3N).
//   Wells: nw wells; well w is water injector (type 0) or producer (type 1),
//   bottom-hole pressure bhp[w] at reference depth dref[w], perforated in
//   cells perf_cells[perf_ptr[w] .. perf_ptr[w+1]) with indices wi[...].
// Returns 0, or -1 on a non-positive pore volume or formation volume factor.
int bg_assemble(const bg_grid* g, const bg_fluid* f,
                const double* kx, const double* ky, const double* kz,
                const double* phi0, const double* depth,
                const double* x, const double* xn, double dt,
                int32_t nw, const int32_t* wtype, const double* bhp, const double* dref,
                const int32_t* perf_ptr, const int32_t* perf_cells, const double* perf_wi,
                const bg_bc* bc,
                const int32_t* rowptr, const int32_t* col, double* R, double* val) {
  const int64_t nx = g->nx, ny = g->ny, nz = g->nz, N = nx * ny * nz;
  const double V = g->dx * g->dy * g->dz;
  std::memset(R, 0, sizeof(double) * 3 * N);
  if (val) std::memset(val, 0, sizeof(double) * 9 * (size_t)rowptr[N]);
  Assembler as{*g, *f, N, rowptr, col, R, val};

  std::vector<Props> P(N);
  for (int64_t c = 0; c < N; ++c) {
    P[c] = cell_props(*f, phi0[c], x[3 * c], x[3 * c + 1], x[3 * c + 2]);
    if (P[c].phi.v <= 0 || P[c].bw.v <= 0 || P[c].bo.v <= 0 || P[c].bg.v <= 0) return -1;
  }

  // accumulation
  for (int64_t c = 0; c < N; ++c) add_accumulation(as, *f, P[c], phi0[c], xn + 3 * c, V, dt, c, R);

  // interior faces (no-flow on the outer faces)
  auto face = [&](int64_t a, int64_t b, double T) { add_face(as, P, x, depth[a], depth[b], a, b, T, R); };

  auto tpfa = [&](double area, double h, double k1, double k2) {
    return kDarcy * area * 2.0 / (h / k1 + h / k2);
  };
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        const int64_t c = i + nx * (j + ny * k);
        if (i < nx - 1) face(c, c + 1, tpfa(g->dy * g->dz, g->dx, kx[c], kx[c + 1]));
        if (j < ny - 1) face(c, c + nx, tpfa(g->dx * g->dz, g->dy, ky[c], ky[c + nx]));
        if (k < nz - 1) face(c, c + nx * ny, tpfa(g->dx * g->dy, g->dz, kz[c], kz[c + nx * ny]));
      }

  // test-only Dirichlet x faces
  if (bc && bc->enabled) {
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j)
        for (int side = 0; side < 2; ++side) {
          const int64_t i = side == 0 ? 0 : nx - 1;
          const int64_t c = i + nx * (j + ny * k);
          const double Tb = kDarcy * g->dy * g->dz * kx[c] / (0.5 * g->dx);
          const double pb = side == 0 ? bc->p_left : bc->p_right;
          Dual<3> dp = pb - Dual<3>::var(x[3 * c], 0);
          Dual<3> fo = Tb * P[c].lo * dp, fw = Tb * P[c].lw * dp;
          Dual<3> fg = Tb * (P[c].rs * P[c].lo + P[c].lg) * dp;
          const Dual<3>* F[3] = {&fo, &fw, &fg};
          double blk[3][3];
          for (int comp = 0; comp < 3; ++comp) {
            R[3 * c + comp] -= F[comp]->v;
            for (int u = 0; u < 3; ++u) blk[comp][u] = -F[comp]->d[u];
          }
          as.add_block(c, c, blk);
        }
  }

  add_wells(as, P, x, depth, nw, wtype, bhp, dref, perf_ptr, perf_cells, perf_wi, R);
  return 0;
}

}  // extern "C"

extern "C" {

// Block pattern of the dual-porosity system (paper Sec. 2.1's dual-porosity
// model): 2N block rows, node c < N the fracture continuum of cell c and node
// N + c its matrix continuum.  Fracture row c holds its 7-point fracture
// neighbours and its matrix node (ascending columns); matrix row N + c holds
// (c, N + c).  nnzb = nnzb(7-point) + 3 N.
int64_t bg_dual_nnzb(const bg_grid* g) {
  const int64_t N = (int64_t)g->nx * g->ny * g->nz;
  return bg_nnzb(g) + 3 * N;
}

void bg_dual_pattern(const bg_grid* g, int32_t* rowptr, int32_t* col) {
  const int64_t N = (int64_t)g->nx * g->ny * g->nz;
  std::vector<int32_t> rp(N + 1), cl(bg_nnzb(g));
  bg_pattern(g, rp.data(), cl.data());
  int64_t e = 0;
  rowptr[0] = 0;
  for (int64_t c = 0; c < N; ++c) {
    for (int32_t k = rp[c]; k < rp[c + 1]; ++k) col[e++] = cl[k];
    col[e++] = (int32_t)(N + c);
    rowptr[c + 1] = (int32_t)e;
  }
  for (int64_t c = 0; c < N; ++c) {
    col[e++] = (int32_t)c;
    col[e++] = (int32_t)(N + c);
    rowptr[N + c + 1] = (int32_t)e;
  }
}

// Dual-porosity residual and Jacobian.  Per cell c: a fracture node (porosity
// phif, permeabilities kx, ky, kz, 7-point flow among fracture nodes, wells)
// and a matrix node (porosity phim, no matrix-matrix flow) exchanging fluid
// with its fracture node through the Warren-Root transfer
// tau = 0.001127 sigma km V lambda_up (Phi_f - Phi_m) (same depth, so the
// potential difference is the pressure difference).  x, xn: 6N (fracture
// nodes' (p, Sw, Sg) first, then the matrix nodes').  Returns 0 or -1.
int bg_assemble_dual(const bg_grid* g, const bg_fluid* f,
                     const double* kx, const double* ky, const double* kz, const double* km,
                     const double* phif, const double* phim, const double* depth,
                     const double* x, const double* xn, double dt, double sigma,
                     int32_t nw, const int32_t* wtype, const double* bhp, const double* dref,
                     const int32_t* perf_ptr, const int32_t* perf_cells, const double* perf_wi,
                     const int32_t* rowptr, const int32_t* col, double* R, double* val) {
  const int64_t nx = g->nx, ny = g->ny, nz = g->nz, N = nx * ny * nz;
  const double V = g->dx * g->dy * g->dz;
  std::memset(R, 0, sizeof(double) * 6 * N);
  if (val) std::memset(val, 0, sizeof(double) * 9 * (size_t)rowptr[2 * N]);
  Assembler as{*g, *f, 2 * N, rowptr, col, R, val};
  std::vector<Props> P(2 * N);
  for (int64_t c = 0; c < 2 * N; ++c) {
    const double ph = c < N ? phif[c] : phim[c - N];
    P[c] = cell_props(*f, ph, x[3 * c], x[3 * c + 1], x[3 * c + 2]);
    if (P[c].phi.v <= 0 || P[c].bw.v <= 0 || P[c].bo.v <= 0 || P[c].bg.v <= 0) return -1;
  }
  for (int64_t c = 0; c < 2 * N; ++c)
    add_accumulation(as, *f, P[c], c < N ? phif[c] : phim[c - N], xn + 3 * c, V, dt, c, R);
  auto tpfa = [&](double area, double h, double k1, double k2) { return kDarcy * area * 2.0 / (h / k1 + h / k2); };
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        const int64_t c = i + nx * (j + ny * k);
        if (i < nx - 1) add_face(as, P, x, depth[c], depth[c + 1], c, c + 1, tpfa(g->dy * g->dz, g->dx, kx[c], kx[c + 1]), R);
        if (j < ny - 1)
          add_face(as, P, x, depth[c], depth[c + nx], c, c + nx, tpfa(g->dx * g->dz, g->dy, ky[c], ky[c + nx]), R);
        if (k < nz - 1)
          add_face(as, P, x, depth[c], depth[c + nx * ny], c, c + nx * ny,
                   tpfa(g->dx * g->dy, g->dz, kz[c], kz[c + nx * ny]), R);
      }
  for (int64_t c = 0; c < N; ++c) add_face(as, P, x, depth[c], depth[c], c, N + c, kDarcy * sigma * km[c] * V, R);
  add_wells(as, P, x, depth, nw, wtype, bhp, dref, perf_ptr, perf_cells, perf_wi, R);
  return 0;
}

}  // extern "C"

namespace {
// a cell-local dual lifted into the well's slots: (p, Sw, Sg) then p_h
Dual<4> lift4(const Dual<3>& a) {
  Dual<4> r(a.v);
  for (int i = 0; i < 3; ++i) r.d[i] = a.d[i];
  return r;
}
}  // namespace

extern "C" {

// Rate-controlled wells (paper Sec. 2.3): a well under a fixed water (ctrl 1),
// oil (ctrl 2) or liquid (ctrl 3) rate has its bottom-hole pressure p_h as an
// unknown and the constraint sum_m Q_ctrl,m(x, p_h) = rate, Q the component
// rates into the perforated nodes of add_wells (stb/day; rate > 0 injects,
// rate < 0 produces).  These wells' perforation terms enter R and the
// diagonal blocks through bg_assemble with bhp[w] = the current p_h; this
// function gives the border of the Newton system (paper Sec. 3.2's A_pw, A_wp,
// A_ww), for the rate-controlled wells in well order (index v) and their
// perforations in order (index e):
//   Rw[v]         = sum_m Q_ctrl,m - rate[w]              (the well's residual)
//   apw[3 e + c]  = dR_c,cell(e) / dp_h = -dQ_c / dp_h     (cell rows, well column)
//   awp[3 e + u]  = dRw[v] / dx_cell(e),u                  (well row, cell columns)
//   aww[v]        = dRw[v] / dp_h
// ctrl[w] = 0 marks a fixed-BHP well (no unknown, skipped).  Returns the
// number of rate-controlled wells, or -2 for an injector (type 0) under an
// oil-rate control (its constraint would not depend on p_h).
int bg_well_border(const bg_fluid* f, const double* phi0, const double* depth, const double* x, int32_t nw,
                   const int32_t* wtype, const int32_t* ctrl, const double* rate, const double* bhp,
                   const double* dref, const int32_t* perf_ptr, const int32_t* perf_cells, const double* perf_wi,
                   double* Rw, double* apw, double* awp, double* aww) {
  int v = 0;
  int64_t e = 0;
  for (int32_t w = 0; w < nw; ++w) {
    if (ctrl[w] == 0) continue;
    if (wtype[w] == 0 && ctrl[w] == 2) return -2;
    Dual<4> total(0.0);
    for (int32_t k = perf_ptr[w]; k < perf_ptr[w + 1]; ++k, ++e) {
      const int64_t c = perf_cells[k];
      const Props C = cell_props(*f, phi0[c], x[3 * c], x[3 * c + 1], x[3 * c + 2]);
      const double WI = perf_wi[k];
      const Dual<4> ph = Dual<4>::var(bhp[w], 3);
      Dual<4> p = lift4(Dual<3>::var(x[3 * c], 0));
      const double dzh = dref[w] - depth[c];
      const Dual<4> dpo = ph - p - lift4(C.go) * dzh;
      const Dual<4> dpw = ph - p - lift4(C.gw) * dzh;
      const Dual<4> dpg = ph - p - lift4(C.gg) * dzh;
      Dual<4> qo(0.0), qw(0.0), qg(0.0);
      if (wtype[w] == 0) {
        qw = WI * lift4(C.lt_res_w) * dpw;
      } else {
        qo = WI * lift4(C.lo) * dpo;
        qw = WI * lift4(C.lw) * dpw;
        qg = WI * (lift4(C.rs) * lift4(C.lo) * dpo + lift4(C.lg) * dpg);
      }
      const Dual<4>* Q[3] = {&qo, &qw, &qg};
      for (int comp = 0; comp < 3; ++comp) apw[3 * e + comp] = -Q[comp]->d[3];
      const Dual<4> qc = ctrl[w] == 1 ? qw : ctrl[w] == 2 ? qo : qo + qw;
      for (int u = 0; u < 3; ++u) awp[3 * e + u] = qc.d[u];
      total = total + qc;
    }
    Rw[v] = total.v - rate[w];
    aww[v] = total.d[3];
    ++v;
  }
  return v;
}

}  // extern "C"
