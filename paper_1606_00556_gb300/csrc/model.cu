// The black-oil residual and Jacobian on the device, and the inexact Newton
// method around the solver (paper Sec. 2.1 Eq. 3 and its closure relations,
// Sec. 2.3 Eq. 4, Sec. 3.1 Alg. 1 with the forcing terms).
//
// Per cell c and component (oil, water, gas):
//   R_c = V / (5.615 dt) [M_c(x) - M_c(x^n)]
//         - sum_faces T sum_phases (x_phase lambda)_upstream (Phi_b - Phi_a)
//         - Q_c (wells at fixed bottom-hole pressure)
// with M_w = phi Sw / Bw, M_o = phi So / Bo, M_g = phi (Sg / Bg + Rs So / Bo);
// mobilities lambda = k_r / (mu B) (Corey two-phase curves, Stone II for the
// oil); potentials Phi = p - rho g D / 144 with the face density the mean of
// its two cells; two-point transmissibilities T = 0.001127 A 2 / (h / k_a +
// h / k_b); phase-potential upwinding (a tie goes to the lower cell index).
// Newton convention: b = -R(x), A = dR/dx.  The derivatives are exact:
// forward-mode dual numbers with the 3 unknowns of a cell, or the 6 of the
// two cells of a face.
//
// Three kernels, no atomics (every sum is in a fixed order):
//   k_cell_props  per cell: the properties the faces need (mobilities and
//                 gravity gradients with their derivatives), the
//                 accumulation term and the cell's well terms;
//   k_faces       per face (one family of x, y or z faces per launch): the
//                 three component fluxes and their derivative blocks with
//                 respect to both cells;
//   k_gather      per cell: residual, b = -R, and the block row of A in BSR
//                 order (columns -z, -y, -x, diag, +x, +y, +z).
// The Jacobian goes into the caller's matrix through the ingest kernel
// (bo_mat_update_values with device values), so the solver sees exactly
// what a host-assembled Jacobian would give it.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "bo_internal.cuh"

namespace bo {
namespace {

constexpr double kDarcyC = 0.001127;  // bbl cp / (day ft^2 psi mD)
constexpr double kFt3PerBbl = 5.615;

// ---- forward-mode dual numbers with K derivative slots
template <int K>
struct Dn {
  double v;
  double d[K];
};
template <int K>
__device__ __forceinline__ Dn<K> dn_const(double a) {
  Dn<K> r;
  r.v = a;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = 0.0;
  return r;
}
template <int K>
__device__ __forceinline__ Dn<K> dn_var(double a, int slot) {
  Dn<K> r = dn_const<K>(a);
  r.d[slot] = 1.0;
  return r;
}
template <int K>
__device__ __forceinline__ Dn<K> operator+(const Dn<K>& a, const Dn<K>& b) {
  Dn<K> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int K>
__device__ __forceinline__ Dn<K> operator-(const Dn<K>& a, const Dn<K>& b) {
  Dn<K> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int K>
__device__ __forceinline__ Dn<K> operator*(const Dn<K>& a, const Dn<K>& b) {
  Dn<K> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int K>
__device__ __forceinline__ Dn<K> operator/(const Dn<K>& a, const Dn<K>& b) {
  Dn<K> r;
  const double inv = 1.0 / b.v;
  r.v = a.v * inv;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * inv;
  return r;
}
template <int K>
__device__ __forceinline__ Dn<K> operator/(double a, const Dn<K>& b) {
  Dn<K> r;
  const double inv = 1.0 / b.v;
  r.v = a * inv;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = -r.v * b.d[i] * inv;
  return r;
}
template <int K>
__device__ __forceinline__ Dn<K> operator*(double s, const Dn<K>& a) {
  Dn<K> r;
  r.v = s * a.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = s * a.d[i];
  return r;
}
template <int K>
__device__ __forceinline__ Dn<K> operator+(double s, const Dn<K>& a) {
  Dn<K> r = a;
  r.v = s + a.v;
  return r;
}
template <int K>
__device__ __forceinline__ Dn<K> operator-(double s, const Dn<K>& a) {
  Dn<K> r;
  r.v = s - a.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = -a.d[i];
  return r;
}
// a cell's dual placed in the slots `off` .. off + 2 of a face dual
__device__ __forceinline__ Dn<6> to_face(const Dn<3>& a, int off) {
  Dn<6> r = dn_const<6>(a.v);
  r.d[off] = a.d[0];
  r.d[off + 1] = a.d[1];
  r.d[off + 2] = a.d[2];
  return r;
}
template <int K>
__device__ __forceinline__ Dn<K> pos_part(const Dn<K>& a) {
  return a.v > 0.0 ? a : dn_const<K>(0.0);
}
// s^e for a normalised saturation s >= 0 (Corey curve): the square exactly
// when e = 2, else pow
template <int K>
__device__ __forceinline__ Dn<K> corey(const Dn<K>& s, double e) {
  if (e == 2.0) return s * s;
  Dn<K> r = dn_const<K>(pow(s.v, e));
  const double dv = s.v > 0.0 ? e * pow(s.v, e - 1.0) : 0.0;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = dv * s.d[i];
  return r;
}

// Relative permeabilities: Corey two-phase curves and the Stone II oil
// relative permeability k_ro = k_rocw [(k_row / k_rocw + k_rw)(k_rog / k_rocw
// + k_rg) - k_rw - k_rg], clamped at 0 (paper Sec. 2.1).
template <int K>
__device__ void rel_perms(const bo_fluid& f, const Dn<K>& sw, const Dn<K>& sg, Dn<K>& krw, Dn<K>& kro, Dn<K>& krg) {
  const double span_w = 1.0 - f.swc - f.sorw;
  const double span_g = 1.0 - f.swc - f.sorg - f.sgc;
  krw = corey(pos_part((1.0 / span_w) * (sw - dn_const<K>(f.swc))), f.nw);
  const Dn<K> krow = corey(pos_part((1.0 / span_w) * ((1.0 - f.sorw) - sw)), f.now);
  krg = corey(pos_part((1.0 / span_g) * (sg - dn_const<K>(f.sgc))), f.ng);
  const Dn<K> krog = corey(pos_part((1.0 / span_g) * ((1.0 - f.swc - f.sorg) - sg)), f.nog);
  const double krocw = pow(fmax(0.0, (1.0 - f.swc - f.sorw) / span_w), f.now);
  const double ic = 1.0 / krocw;
  kro = pos_part(krocw * ((ic * krow + krw) * (ic * krog + krg) - krw - krg));
}

// The cell quantities of Eq. 3 as functions of (p, Sw, Sg): the face
// quantities (mobilities lo, lw, lg, Rs lo and gravity gradients go, gw, gg,
// when lo is non-NULL), the total mobility over Bw, the component amounts per
// bulk volume, and (chk) phi, Bw, Bo, Bg for the validity check.
template <int K>
__device__ void cell_quantities(const bo_fluid& f, double phi0, const Dn<K>& p, const Dn<K>& sw, const Dn<K>& sg,
                                Dn<K>* lo, Dn<K>* lw, Dn<K>* lg, Dn<K>* rso, Dn<K>* go, Dn<K>* gw, Dn<K>* gg,
                                Dn<K>* lt_w, Dn<K>* mo, Dn<K>* mw, Dn<K>* mg, double* chk) {
  const Dn<K> dp = p - dn_const<K>(f.pref);
  const Dn<K> phi = phi0 * (1.0 + f.cr * dp);
  const Dn<K> bw = f.bw0 * (1.0 - f.cw * dp);
  const Dn<K> bo = f.bo0 + f.dbo * dp;
  const Dn<K> rs = f.rs0 + f.drs * dp;
  const Dn<K> bg = f.bg0 - f.dbg * dp;
  const Dn<K> so = 1.0 - (sw + sg);
  Dn<K> krw, kro, krg;
  rel_perms(f, sw, sg, krw, kro, krg);
  if (lo) {
    *lo = kro / (f.muo * bo);
    *lw = krw / (f.muw * bw);
    *lg = krg / (f.mug * bg);
    *rso = rs * *lo;
    *lt_w = ((1.0 / f.muw) * krw + (1.0 / f.muo) * kro + (1.0 / f.mug) * krg) / bw;
    // reservoir densities (lb / ft^3) over 144 in^2 / ft^2
    const double gas_sc = 1000.0 * f.rhog_sc;  // lb of gas in one Mscf
    *gw = (f.gravity * f.rhow_sc / 144.0) * (1.0 / bw);
    *go = (f.gravity / (144.0 * kFt3PerBbl)) * ((f.rhoo_sc * kFt3PerBbl + gas_sc * rs) / bo);
    *gg = (f.gravity * gas_sc / (144.0 * kFt3PerBbl)) * (1.0 / bg);
  }
  *mw = phi * sw / bw;
  *mo = phi * so / bo;
  *mg = phi * (sg / bg + rs * so / bo);
  if (chk) {
    chk[0] = phi.v;
    chk[1] = bw.v;
    chk[2] = bo.v;
    chk[3] = bg.v;
  }
}

}  // namespace
}  // namespace bo

struct bo_model {
  bo_ctx* ctx;
  bo_grid grid;
  bo::Geom g;
  bo_fluid fluid;
  int64_t N, nnzb;
  double* kx;
  double* ky;
  double* kz;
  double* phi0;
  double* depth;
  int32_t* cperf_ptr;  // N + 1: perforations of each cell
  double* cperf;       // per perforation of a cell (cell order): (type, bhp, dref, WI)
  int64_t nperf;
  int32_t* rowptr;     // BSR row pointers of the 7-point pattern
  double* props;       // 28 N
  double* racc;        // 3 N accumulation + well residual
  double* dacc;        // 9 N accumulation + well diagonal block
  double* face;        // 3 families x 21 x N: flux (3), d/da (9), d/db (9)
  double* val;         // 9 nnzb Jacobian in BSR order
  double* b;           // 3 N right-hand side of the last assembly
  double* r;           // 3 N linear residual (Newton)
  double* dx;          // 3 N Newton update
  double* partials;    // reductions
  double* red;         // reduction results (device)
  double* h_red;       // pinned host copy
  unsigned* counter;
  int* err;
};

namespace bo {
namespace {

constexpr int kQ = 7;  // face quantities per cell: lo, lw, lg, rso, go, gw, gg

// per cell: face quantities, accumulation and wells
__global__ void __launch_bounds__(kThreads) k_cell_props(Geom g, bo_fluid f, double dx, double dy, double dz,
                                                        const double* __restrict__ phi0, const double* __restrict__ depth,
                                                        const double* __restrict__ x, const double* __restrict__ xn,
                                                        double dt, const int32_t* __restrict__ cperf_ptr,
                                                        const double* __restrict__ cperf, double* __restrict__ props,
                                                        double* __restrict__ racc, double* __restrict__ dacc,
                                                        int* err) {
  wait_prior_grid();
  const double scale = dx * dy * dz / (kFt3PerBbl * dt);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.N; c += (int64_t)gridDim.x * blockDim.x) {
    const Dn<3> p = dn_var<3>(x[3 * c], 0), sw = dn_var<3>(x[3 * c + 1], 1), sg = dn_var<3>(x[3 * c + 2], 2);
    Dn<3> Q[kQ], ltw, mo, mw, mg;
    double chk[4];
    cell_quantities<3>(f, phi0[c], p, sw, sg, &Q[0], &Q[1], &Q[2], &Q[3], &Q[4], &Q[5], &Q[6], &ltw, &mo, &mw, &mg,
                       chk);
    if (!(chk[0] > 0.0 && chk[1] > 0.0 && chk[2] > 0.0 && chk[3] > 0.0)) atomicOr(err, kErrBreakdown);
#pragma unroll
    for (int k = 0; k < kQ; ++k) {
      props[(size_t)(4 * k) * g.N + c] = Q[k].v;
#pragma unroll
      for (int u = 0; u < 3; ++u) props[(size_t)(4 * k + 1 + u) * g.N + c] = Q[k].d[u];
    }
    // the previous time level's amounts (values only)
    const Dn<1> pn = dn_const<1>(xn[3 * c]), swn = dn_const<1>(xn[3 * c + 1]), sgn = dn_const<1>(xn[3 * c + 2]);
    Dn<1> mon, mwn, mgn;
    cell_quantities<1>(f, phi0[c], pn, swn, sgn, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                       nullptr, &mon, &mwn, &mgn, nullptr);
    const Dn<3>* M[3] = {&mo, &mw, &mg};
    const double Mn[3] = {mon.v, mwn.v, mgn.v};
    double R[3], D[9];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      R[e] = scale * (M[e]->v - Mn[e]);
#pragma unroll
      for (int u = 0; u < 3; ++u) D[3 * e + u] = scale * M[e]->d[u];
    }
    // wells at fixed bottom-hole pressure (Eq. 4): rate into the cell
    // WI lambda (p_bh - p - grad (z_ref - z)); a water injector with the
    // cell's total mobility, a producer with the phase mobilities
    for (int32_t e = cperf_ptr[c]; e < cperf_ptr[c + 1]; ++e) {
      const double type = cperf[4 * (size_t)e], bhp = cperf[4 * (size_t)e + 1], dref = cperf[4 * (size_t)e + 2],
                   wi = cperf[4 * (size_t)e + 3];
      const double dzh = dref - depth[c];
      Dn<3> q[3];
      if (type == 0.0) {
        q[0] = dn_const<3>(0.0);
        q[2] = dn_const<3>(0.0);
        q[1] = wi * (ltw * ((bhp - p) - dzh * Q[5]));
      } else {
        const Dn<3> dpo = (bhp - p) - dzh * Q[4];
        q[0] = wi * (Q[0] * dpo);
        q[1] = wi * (Q[1] * ((bhp - p) - dzh * Q[5]));
        q[2] = wi * (Q[3] * dpo + Q[2] * ((bhp - p) - dzh * Q[6]));
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        R[r] -= q[r].v;
#pragma unroll
        for (int u = 0; u < 3; ++u) D[3 * r + u] -= q[r].d[u];
      }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) racc[(size_t)r * g.N + c] = R[r];
#pragma unroll
    for (int k = 0; k < 9; ++k) dacc[(size_t)k * g.N + c] = D[k];
  }
}

__device__ __forceinline__ Dn<3> load_q(const double* __restrict__ props, int64_t N, int k, int64_t c) {
  Dn<3> r;
  r.v = props[(size_t)(4 * k) * N + c];
  r.d[0] = props[(size_t)(4 * k + 1) * N + c];
  r.d[1] = props[(size_t)(4 * k + 2) * N + c];
  r.d[2] = props[(size_t)(4 * k + 3) * N + c];
  return r;
}

// The three component fluxes from cell b into cell a through the face
// (a, b = a + stride), b the larger index, and their derivatives: slots 0-2
// a's unknowns, 3-5 b's.  fam 0: x faces, 1: y, 2: z; a face exists where a
// is not on the family's last grid plane.
__global__ void __launch_bounds__(kThreads) k_faces(Geom g, int fam, double area, double h,
                                                   const double* __restrict__ perm, const double* __restrict__ depth,
                                                   const double* __restrict__ x, const double* __restrict__ props,
                                                   double* __restrict__ out) {
  wait_prior_grid();
  const int64_t stride = fam == 0 ? 1 : fam == 1 ? (int64_t)g.nx : (int64_t)g.nx * g.ny;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < g.N; a += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = a / g.nx;
    const int i = (int)(a - row * g.nx), j = (int)(row % g.ny), k = (int)(row / g.ny);
    const bool has = fam == 0 ? i < g.nx - 1 : fam == 1 ? j < g.ny - 1 : k < g.nz - 1;
    if (!has) continue;
    const int64_t b = a + stride;
    const double T = kDarcyC * area * 2.0 / (h / perm[a] + h / perm[b]);
    const double dzab = depth[b] - depth[a];
    const Dn<6> dpab = dn_var<6>(x[3 * b], 3) - dn_var<6>(x[3 * a], 0);
    Dn<6> dphi[3];  // oil, water, gas potential differences Phi_b - Phi_a
#pragma unroll
    for (int ph = 0; ph < 3; ++ph) {
      const int qk = 4 + ph;  // go, gw, gg
      const Dn<6> grad = to_face(load_q(props, g.N, qk, a), 0) + to_face(load_q(props, g.N, qk, b), 3);
      dphi[ph] = dpab - (0.5 * dzab) * grad;
    }
    // upstream quantity: b's where Phi_b > Phi_a, a's where lower; a tie
    // goes to a, the lower index
    auto up = [&](const Dn<6>& d, int qk) {
      return d.v > 0.0 ? to_face(load_q(props, g.N, qk, b), 3) : to_face(load_q(props, g.N, qk, a), 0);
    };
    const Dn<6> fo = T * (up(dphi[0], 0) * dphi[0]);
    const Dn<6> fw = T * (up(dphi[1], 1) * dphi[1]);
    const Dn<6> fg = T * (up(dphi[0], 3) * dphi[0] + up(dphi[2], 2) * dphi[2]);
    const Dn<6>* F[3] = {&fo, &fw, &fg};
    double* o = out + (size_t)fam * 21 * g.N;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      o[(size_t)r * g.N + a] = F[r]->v;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        o[(size_t)(3 + 3 * r + u) * g.N + a] = F[r]->d[u];
        o[(size_t)(12 + 3 * r + u) * g.N + a] = F[r]->d[3 + u];
      }
    }
  }
}

// Per cell: R = accumulation and wells - (fluxes in), b = -R, and the block
// row in BSR order.  A face (a, b) adds -F to a's residual and +F to b's;
// its derivative blocks go to a's row as -dF/da (diagonal), -dF/db (column
// b), and to b's row as dF/da (column a), dF/db (diagonal).
__global__ void __launch_bounds__(kThreads) k_gather(Geom g, const int32_t* __restrict__ rowptr,
                                                    const double* __restrict__ racc, const double* __restrict__ dacc,
                                                    const double* __restrict__ face, double* __restrict__ bvec,
                                                    double* __restrict__ val) {
  wait_prior_grid();
  const int64_t strides[3] = {1, (int64_t)g.nx, (int64_t)g.nx * g.ny};
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.N; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = c / g.nx;
    const int i = (int)(c - row * g.nx), j = (int)(row % g.ny), k = (int)(row / g.ny);
    const int lo[3] = {i > 0, j > 0, k > 0};
    const int hi[3] = {i < g.nx - 1, j < g.ny - 1, k < g.nz - 1};
    double R[3], D[9];
#pragma unroll
    for (int r = 0; r < 3; ++r) R[r] = racc[(size_t)r * g.N + c];
#pragma unroll
    for (int e = 0; e < 9; ++e) D[e] = dacc[(size_t)e * g.N + c];
    double off[6][9];  // blocks of the neighbours: -z, -y, -x, +x, +y, +z
    // faces where c is the higher cell: (c - stride, c)
#pragma unroll
    for (int fam = 2; fam >= 0; --fam) {
      const int slot = 2 - fam;  // -z: 0, -y: 1, -x: 2
      if (!lo[fam]) continue;
      const int64_t a = c - strides[fam];
      const double* o = face + (size_t)fam * 21 * g.N;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        R[r] += o[(size_t)r * g.N + a];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          off[slot][3 * r + u] = o[(size_t)(3 + 3 * r + u) * g.N + a];
          D[3 * r + u] += o[(size_t)(12 + 3 * r + u) * g.N + a];
        }
      }
    }
    // faces where c is the lower cell: (c, c + stride)
#pragma unroll
    for (int fam = 0; fam < 3; ++fam) {
      const int slot = 3 + fam;  // +x: 3, +y: 4, +z: 5
      if (!hi[fam]) continue;
      const double* o = face + (size_t)fam * 21 * g.N;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        R[r] -= o[(size_t)r * g.N + c];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          D[3 * r + u] -= o[(size_t)(3 + 3 * r + u) * g.N + c];
          off[slot][3 * r + u] = -o[(size_t)(12 + 3 * r + u) * g.N + c];
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) bvec[3 * c + r] = -R[r];
    double* v = val + 9 * (size_t)rowptr[c];
    auto put = [&](const double* blk) {
#pragma unroll
      for (int e = 0; e < 9; ++e) v[e] = blk[e];
      v += 9;
    };
    if (lo[2]) put(off[0]);
    if (lo[1]) put(off[1]);
    if (lo[0]) put(off[2]);
    put(D);
    if (hi[0]) put(off[3]);
    if (hi[1]) put(off[4]);
    if (hi[2]) put(off[5]);
  }
}

// out[0] = ||u||^2 (or ||u - v||^2 with v non-NULL), deterministic:
// per-block partials summed by the last block
__global__ void __launch_bounds__(kThreads) k_sqnorm(int64_t n, const double* __restrict__ u,
                                                    const double* __restrict__ v, double* partials,
                                                    unsigned* counter, double* out) {
  wait_prior_grid();
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = v ? u[i] - v[i] : u[i];
    acc = fma(d, d, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  if (!last_block(counter, gridDim.x)) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(partials + i);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    *out = s;
    *counter = 0;
  }
}

__global__ void k_copy64(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
  wait_prior_grid();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

constexpr int kNormBlocks = 2 * 152;

// ||u|| or ||u - v|| on the model's stream (synchronises)
int model_norm(bo_model* M, int64_t n, const double* u, const double* v, double* out) {
  cudaStream_t s = M->ctx->stream;
  (launch_pdl(k_sqnorm, kNormBlocks, kThreads, 0, s, n, u, v, M->partials, M->counter, M->red), note_launch());
  if (cudaMemcpyAsync(M->h_red, M->red, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BO_ERR_CUDA;
  *out = std::sqrt(*M->h_red);
  return BO_OK;
}

int model_assemble(bo_model* M, const double* x, const double* xn, double dt) {
  cudaStream_t s = M->ctx->stream;
  const Geom& g = M->g;
  const bo_grid& gr = M->grid;
  cudaMemsetAsync(M->err, 0, sizeof(int), s);
  const int gc = grid_for(g.N);
  (launch_pdl(k_cell_props, gc, kThreads, 0, s, g, M->fluid, gr.dx, gr.dy, gr.dz, M->phi0, M->depth, x, xn, dt,
      M->cperf_ptr, M->cperf, M->props, M->racc, M->dacc, M->err),
   note_launch());
  (launch_pdl(k_faces, gc, kThreads, 0, s, g, 0, gr.dy * gr.dz, gr.dx, M->kx, M->depth, x, M->props, M->face), note_launch());
  (launch_pdl(k_faces, gc, kThreads, 0, s, g, 1, gr.dx * gr.dz, gr.dy, M->ky, M->depth, x, M->props, M->face), note_launch());
  (launch_pdl(k_faces, gc, kThreads, 0, s, g, 2, gr.dx * gr.dy, gr.dz, M->kz, M->depth, x, M->props, M->face), note_launch());
  (launch_pdl(k_gather, gc, kThreads, 0, s, g, M->rowptr, M->racc, M->dacc, M->face, M->b, M->val), note_launch());
  int h = 0;
  if (cudaMemcpyAsync(&h, M->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BO_ERR_CUDA;
  return h ? BO_ERR_BREAKDOWN : BO_OK;
}

void model_free(bo_model* M) {
  auto fr = [](void* p) { if (p) cudaFree(p); };
  fr(M->kx); fr(M->ky); fr(M->kz); fr(M->phi0); fr(M->depth); fr(M->cperf_ptr); fr(M->cperf); fr(M->rowptr);
  fr(M->props); fr(M->racc); fr(M->dacc); fr(M->face); fr(M->val); fr(M->b); fr(M->r); fr(M->dx);
  fr(M->partials); fr(M->red); fr(M->counter); fr(M->err);
  if (M->h_red) cudaFreeHost(M->h_red);
}

}  // namespace
}  // namespace bo

extern "C" {

void bo_newton_opts_default(bo_newton_opts* o) {
  if (!o) return;
  o->eps = 0.0;
  o->eps_rel = 1e-8;
  o->forcing = BO_FORCING_EW3;
  o->theta_fixed = 1e-2;
  o->theta_max = 0.1;
  o->theta_min = 1e-10;
  o->gamma = 0.9;
  o->beta = 2.0;
  o->maxit = 20;
  o->restart = 30;
  o->lin_maxit = 1000;
}

int bo_model_create(bo_ctx* ctx, const bo_grid* grid, const bo_fluid* fluid, const double* kx, const double* ky,
                    const double* kz, const double* phi0, const double* depth, int32_t nperf,
                    const int32_t* perf_cell, const int32_t* perf_type, const double* perf_bhp,
                    const double* perf_dref, const double* perf_wi, bo_model** out) {
  using namespace bo;
  if (!ctx || !grid || !fluid || !kx || !ky || !kz || !phi0 || !depth || !out || nperf < 0) return BO_ERR_ARG;
  if (nperf > 0 && (!perf_cell || !perf_type || !perf_bhp || !perf_dref || !perf_wi)) return BO_ERR_ARG;
  if (grid->nx < 2 || grid->ny < 1 || grid->nz < 1 || (grid->nx % 2) != 0 || grid->ncontinua != 1 ||
      (int64_t)grid->nx * grid->ny * grid->nz > ((int64_t)1 << 28))
    return BO_ERR_ARG;
  if (!(grid->dx > 0 && grid->dy > 0 && grid->dz > 0)) return BO_ERR_ARG;
  const int64_t N = (int64_t)grid->nx * grid->ny * grid->nz;
  for (int32_t e = 0; e < nperf; ++e)
    if (perf_cell[e] < 0 || perf_cell[e] >= N || (perf_type[e] != 0 && perf_type[e] != 1) || !std::isfinite(perf_wi[e]))
      return BO_ERR_ARG;
  for (int64_t c = 0; c < N; ++c)
    if (!(kx[c] > 0 && ky[c] > 0 && kz[c] > 0 && phi0[c] > 0) || !std::isfinite(depth[c])) return BO_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  bo_model* M = new (std::nothrow) bo_model();
  if (!M) return BO_ERR_OOM;
  M->ctx = ctx;
  M->grid = *grid;
  M->fluid = *fluid;
  M->N = N;
  const int64_t nx = grid->nx, ny = grid->ny, nz = grid->nz;
  M->nnzb = N + 2 * ((nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1));
  M->g = Geom{grid->nx, grid->ny, grid->nz, grid->nx / 2, N, N / 2};
  // perforations grouped by cell (the order within a cell: as given)
  std::vector<int32_t> cptr(N + 1, 0);
  for (int32_t e = 0; e < nperf; ++e) cptr[perf_cell[e] + 1]++;
  for (int64_t c = 0; c < N; ++c) cptr[c + 1] += cptr[c];
  std::vector<double> cp(4 * (size_t)std::max<int32_t>(nperf, 1), 0.0);
  {
    std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
    for (int32_t e = 0; e < nperf; ++e) {
      const int32_t at = fill[perf_cell[e]]++;
      cp[4 * (size_t)at] = perf_type[e];
      cp[4 * (size_t)at + 1] = perf_bhp[e];
      cp[4 * (size_t)at + 2] = perf_dref[e];
      cp[4 * (size_t)at + 3] = perf_wi[e];
    }
  }
  // BSR row pointers of the 7-point pattern
  std::vector<int32_t> rp(N + 1, 0);
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        const int64_t c = i + nx * (j + ny * k);
        rp[c + 1] = rp[c] + 1 + (i > 0) + (i < nx - 1) + (j > 0) + (j < ny - 1) + (k > 0) + (k < nz - 1);
      }
  bool ok = true;
  auto al = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (ok && cudaMalloc(&p, bytes) != cudaSuccess) {
      ok = false;
      return nullptr;
    }
    return p;
  };
  const size_t d = sizeof(double);
  M->kx = (double*)al(N * d);
  M->ky = (double*)al(N * d);
  M->kz = (double*)al(N * d);
  M->phi0 = (double*)al(N * d);
  M->depth = (double*)al(N * d);
  M->cperf_ptr = (int32_t*)al((N + 1) * sizeof(int32_t));
  M->cperf = (double*)al(cp.size() * d);
  M->rowptr = (int32_t*)al((N + 1) * sizeof(int32_t));
  M->props = (double*)al((size_t)4 * kQ * N * d);
  M->racc = (double*)al(3 * N * d);
  M->dacc = (double*)al(9 * N * d);
  M->face = (double*)al((size_t)3 * 21 * N * d);
  M->val = (double*)al(9 * (size_t)M->nnzb * d);
  M->b = (double*)al(3 * N * d);
  M->r = (double*)al(3 * N * d);
  M->dx = (double*)al(3 * N * d);
  M->partials = (double*)al(kNormBlocks * d);
  M->red = (double*)al(4 * d);
  M->counter = (unsigned*)al(sizeof(unsigned));
  M->err = (int*)al(sizeof(int));
  if (ok && cudaMallocHost(&M->h_red, 4 * d) != cudaSuccess) ok = false;
  M->nperf = nperf;
  cudaStream_t s = ctx->stream;
  if (ok) {
    cudaMemcpyAsync(M->kx, kx, N * d, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(M->ky, ky, N * d, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(M->kz, kz, N * d, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(M->phi0, phi0, N * d, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(M->depth, depth, N * d, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(M->cperf_ptr, cptr.data(), (N + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(M->cperf, cp.data(), cp.size() * d, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(M->rowptr, rp.data(), (N + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(M->counter, 0, sizeof(unsigned), s);
    if (cudaStreamSynchronize(s) != cudaSuccess) ok = false;
  }
  if (!ok) {
    model_free(M);
    delete M;
    return BO_ERR_OOM;
  }
  ctx->refs++;
  *out = M;
  return BO_OK;
}

int bo_model_destroy(bo_model* M) {
  using namespace bo;
  if (!M) return BO_ERR_ARG;
  cudaSetDevice(M->ctx->device);
  cudaStreamSynchronize(M->ctx->stream);
  bo_ctx* c = M->ctx;
  model_free(M);
  delete M;
  ctx_release_ref(c);
  return BO_OK;
}

int bo_model_assemble(bo_model* M, const double* x, const double* xn, double dt, double* b, double* val,
                      double* bnorm) {
  using namespace bo;
  if (!M || !x || !xn || !(dt > 0.0)) return BO_ERR_ARG;
  if (cudaSetDevice(M->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  int rc = model_assemble(M, x, xn, dt);
  if (rc != BO_OK) return rc;
  cudaStream_t s = M->ctx->stream;
  const int64_t n = 3 * M->N;
  if (b) (launch_pdl(k_copy64, grid_for(n), kThreads, 0, s, n, M->b, b), note_launch());
  if (val) (launch_pdl(k_copy64, grid_for(9 * M->nnzb), kThreads, 0, s, 9 * M->nnzb, M->val, val), note_launch());
  if (bnorm) {
    rc = model_norm(M, n, M->b, nullptr, bnorm);
    if (rc != BO_OK) return rc;
  }
  return cudaStreamSynchronize(s) == cudaSuccess ? BO_OK : BO_ERR_CUDA;
}

int bo_newton_solve(bo_model* M, bo_prec* P, double* x, const double* xn, double dt, const bo_newton_opts* opts,
                    bo_newton_info* info) {
  using namespace bo;
  if (!M || !P || !x || !xn || !(dt > 0.0)) return BO_ERR_ARG;
  bo_mat* A = P->mat;
  if (A->ctx != M->ctx || A->grid.nx != M->grid.nx || A->grid.ny != M->grid.ny || A->grid.nz != M->grid.nz ||
      A->kind != 0)
    return BO_ERR_ARG;
  bo_newton_opts o;
  bo_newton_opts_default(&o);
  if (opts) o = *opts;
  if (o.forcing < BO_FORCING_FIXED || o.forcing > BO_FORCING_EW3 || o.maxit < 0 || o.maxit > BO_NEWTON_MAX_STEPS ||
      !(o.theta_min > 0.0) || !(o.theta_max >= o.theta_min) || o.theta_max >= 1.0 ||
      (o.forcing == BO_FORCING_FIXED && !(o.theta_fixed > 0.0 && o.theta_fixed < 1.0)))
    return BO_ERR_ARG;
  if (cudaSetDevice(M->ctx->device) != cudaSuccess) return BO_ERR_CUDA;
  bo_newton_info inf{};
  cudaStream_t s = M->ctx->stream;
  const int64_t n = 3 * M->N;
  auto finish = [&](int st) {
    inf.status = st;
    if (info) *info = inf;
    return st;
  };
  // b(x^0) and A(x^0)
  int rc = model_assemble(M, x, xn, dt);
  if (rc != BO_OK) return finish(rc);
  double nb = 0.0;
  if ((rc = model_norm(M, n, M->b, nullptr, &nb)) != BO_OK) return finish(rc);
  const double eps = o.eps > 0.0 ? o.eps : o.eps_rel * nb;
  inf.bnorm[0] = nb;
  double theta = o.forcing == BO_FORCING_FIXED ? o.theta_fixed : o.theta_max;
  bo_solve_opts so;
  bo_solve_opts_default(&so);
  so.restart = o.restart;
  so.maxit = o.lin_maxit;
  so.x0_is_zero = 1;
  so.mem = BO_MEM_DEVICE;
  while (nb >= eps && inf.iters < o.maxit) {
    // the Newton system of x^l: A dx = b to ||b - A dx|| <= theta ||b|| (Alg. 1)
    if ((rc = bo_mat_update_values(A, M->val, BO_MEM_DEVICE)) != BO_OK) return finish(rc);
    if ((rc = bo_prec_update(P)) != BO_OK) return finish(rc);
    so.tol = theta;
    bo_solve_info si{};
    rc = bo_solve(P, M->b, M->dx, &so, &si);
    if (rc != BO_OK && rc != BO_ERR_NOT_CONVERGED) return finish(rc);
    // r = b - A dx with this step's A; x^{l+1} = x^l + dx
    (launch_pdl(k_copy64, grid_for(n), kThreads, 0, s, n, M->b, M->r), note_launch());
    launch_spmv_nat(A, -1.0, M->dx, 1.0, M->r, BO_PREC_FP64);
    launch_newton_update(x, M->dx, n, s);
    double nr = 0.0;
    if ((rc = model_norm(M, n, M->r, nullptr, &nr)) != BO_OK) return finish(rc);
    // b(x^{l+1}) and A(x^{l+1}) (r is kept for the first forcing term)
    if ((rc = model_assemble(M, x, xn, dt)) != BO_OK) return finish(rc);
    double nb_new = 0.0, ndiff = 0.0;
    if ((rc = model_norm(M, n, M->b, nullptr, &nb_new)) != BO_OK) return finish(rc);
    if ((rc = model_norm(M, n, M->b, M->r, &ndiff)) != BO_OK) return finish(rc);
    const int l = inf.iters;
    inf.theta[l] = theta;
    inf.lin_iters[l] = si.iters;
    inf.lin_rel_res[l] = nr / nb;
    inf.bnorm[l + 1] = nb_new;
    inf.lin_total += si.iters;
    inf.iters = l + 1;
    // the next forcing term (Sec. 3.1), clipped to [theta_min, theta_max]
    if (o.forcing != BO_FORCING_FIXED) {
      double t = 0.0;
      if (o.forcing == BO_FORCING_EW1) t = ndiff / nb;
      else if (o.forcing == BO_FORCING_EW2) t = std::fabs(nb_new - nr) / nb;
      else t = o.gamma * std::pow(nb_new / nb, o.beta);
      theta = std::min(std::max(t, o.theta_min), o.theta_max);
    }
    nb = nb_new;
    if (!std::isfinite(nb)) return finish(BO_ERR_NONFINITE);
  }
  inf.converged = nb < eps;
  return finish(inf.converged ? BO_OK : BO_ERR_NOT_CONVERGED);
}

}  // extern "C"
