"""Pins of the black-oil Jacobian generator against physics that fixes the
answer independently of the code: symmetric zero-row-sum transmissibility
Laplacian under no-flow (paper Sec. 2.1 boundary condition), per-component
mass balance, exact derivatives vs central differences, the linear pressure
profile of incompressible flow between two constant-pressure faces, Stone II
end-point identities and Peaceman's equivalent radius."""
import numpy as np
import pytest

import bogen
from bogen import BC, Well, incompressible_fluid, default_fluid


def _dense(a):
    nb = a["rowptr"].size - 1
    A = np.zeros((3 * nb, 3 * nb))
    for i in range(nb):
        for e in range(a["rowptr"][i], a["rowptr"][i + 1]):
            j = a["col"][e]
            A[3 * i:3 * i + 3, 3 * j:3 * j + 3] += a["val"][e]
    return A


def _hetero_case(nx=6, ny=5, nz=4, seed=3, fluid=None):
    rng = np.random.default_rng(seed)
    c = bogen.uniform_case(nx, ny, nz, fluid=fluid)
    N = c.N
    c.kx = np.exp(rng.normal(4, 1.0, N))
    c.ky = np.exp(rng.normal(4, 1.0, N))
    c.kz = 0.1 * np.exp(rng.normal(4, 1.0, N))
    return c, rng


def test_pattern_is_seven_point_sorted():
    rowptr, col = bogen.pattern(4, 3, 2)
    N = 24
    for c in range(N):
        cols = col[rowptr[c]:rowptr[c + 1]]
        assert np.all(np.diff(cols) > 0)
        i, j, k = c % 4, (c // 4) % 3, c // 12
        exp = {c}
        if i > 0: exp.add(c - 1)
        if i < 3: exp.add(c + 1)
        if j > 0: exp.add(c - 4)
        if j < 2: exp.add(c + 4)
        if k > 0: exp.add(c - 12)
        if k < 1: exp.add(c + 12)
        assert set(cols.tolist()) == exp


def test_transmissibility_block_symmetric_zero_row_sums():
    # incompressible fluid, uniform saturations, no gravity, no wells: the
    # (oil equation, pressure) entries are lambda_o times the weighted graph
    # Laplacian of the two-point transmissibilities
    c, _ = _hetero_case(fluid=incompressible_fluid())
    a = bogen.assemble(c)
    A = _dense(a)
    T = A[0::3, 0::3]
    scale = np.abs(T).max()
    assert scale > 0
    assert np.abs(T - T.T).max() <= 1e-15 * scale * 10
    assert np.abs(T.sum(axis=1)).max() <= 1e-12 * scale
    # off-diagonals non-positive, diagonal positive (an M-matrix Laplacian)
    off = T - np.diag(np.diag(T))
    assert off.max() <= 0 and np.diag(T).min() > 0


def test_face_transmissibility_is_harmonic():
    c = bogen.uniform_case(2, 1, 1, fluid=incompressible_fluid())
    c.kx = np.array([50.0, 200.0])
    a = bogen.assemble(c)
    A = _dense(a)
    fl = c.fluid
    kro = bogen.relperm(fl, 0.2, 0.05)[1]
    lam_o = kro / (fl.muo * fl.bo0)
    T = 0.001127 * (100.0 * 20.0) / (100.0 / 2 / 50.0 + 100.0 / 2 / 200.0)
    assert A[0, 3] == pytest.approx(-T * lam_o, rel=1e-13)


@pytest.mark.parametrize("with_wells", [False, True])
def test_component_mass_balance(with_wells):
    # summing R over all cells cancels every interior flux: what remains is
    # the accumulation minus the well terms (no-flow outer boundary)
    c, rng = _hetero_case()
    N = c.N
    c.x = c.xn * rng.uniform(0.95, 1.05, 3 * N)
    if with_wells:
        c.wells = [Well(0, 3400.0, np.array([0, 30, 60, 90], np.int32)),
                   Well(1, 2600.0, np.array([29, 59, 89, 119], np.int32))]
    a = bogen.assemble(c)
    V = c.dx * c.dy * c.dz
    acc = np.zeros(3)
    for i in range(N):
        for comp in range(3):
            m1 = bogen.cell_mass(c.fluid, c.phi0[i], *c.x[3 * i:3 * i + 3], comp)
            m0 = bogen.cell_mass(c.fluid, c.phi0[i], *c.xn[3 * i:3 * i + 3], comp)
            acc[comp] += V / (5.615 * c.dt) * (m1 - m0)
    tot = a["R"].reshape(N, 3).sum(axis=0)
    if not with_wells:
        assert np.allclose(tot, acc, rtol=1e-10, atol=1e-9 * np.abs(a["R"]).max())
    else:
        q = acc - tot  # the well terms
        # water injector adds water only; the producer removes oil and gas
        assert q[1] != 0 and q[0] < 0 and q[2] < 0


def test_flux_jacobian_column_sums_vanish():
    # with no accumulation (dt -> infinity) and no wells sum_i R_c,i == 0 for
    # every state, so every column of each component's Jacobian sums to zero
    c, rng = _hetero_case()
    c.dt = 1e30
    c.x = c.xn * rng.uniform(0.95, 1.05, 3 * c.N)
    A = _dense(bogen.assemble(c))
    scale = np.abs(A).max()
    for comp in range(3):
        cs = A[comp::3, :].sum(axis=0)
        assert np.abs(cs).max() <= 1e-11 * scale


def test_exact_jacobian_matches_central_differences():
    c, rng = _hetero_case(nx=4, ny=3, nz=3)
    c.x = c.xn * rng.uniform(0.95, 1.05, 3 * c.N)
    c.wells = [Well(0, 3400.0, np.array([0, 12, 24], np.int32)), Well(1, 2600.0, np.array([11, 23, 35], np.int32))]
    A = _dense(bogen.assemble(c))
    n = 3 * c.N
    J = np.zeros((n, n))
    for u in range(n):
        h = 1e-6 * max(abs(c.x[u]), 1e-3)
        xp = c.x.copy(); xp[u] += h
        xm = c.x.copy(); xm[u] -= h
        J[:, u] = (bogen.assemble(c, jacobian=False, x=xp)["R"] - bogen.assemble(c, jacobian=False, x=xm)["R"]) / (2 * h)
    for u in range(n):
        col_scale = max(np.abs(A[:, u]).max(), 1e-12)
        assert np.abs(J[:, u] - A[:, u]).max() <= 1e-5 * col_scale


def _linear_profile_case(kx_columns):
    nx = len(kx_columns)
    fl = incompressible_fluid()
    c = bogen.uniform_case(nx, 3, 2, fluid=fl)
    c.kx = np.tile(np.asarray(kx_columns, float), 6)
    c.bc = BC(1, 3500.0, 2500.0)
    return c


def test_linear_pressure_profile_homogeneous():
    # incompressible flow between two constant-pressure faces: one Newton
    # step from a uniform state lands on p(x) = pL + (pR - pL) x / L at the
    # cell centres; saturations do not change
    c = _linear_profile_case([100.0] * 10)
    a = bogen.assemble(c)
    dx = np.linalg.solve(_dense(a), a["b"])
    p = c.x[0::3] + dx[0::3]
    xc = (np.arange(10) + 0.5) * c.dx
    exact = 3500.0 + (2500.0 - 3500.0) * xc / (10 * c.dx)
    assert np.abs(p - np.tile(exact, 6)).max() <= 1e-9 * 3500
    assert np.abs(dx[1::3]).max() < 1e-9 and np.abs(dx[2::3]).max() < 1e-9


def test_linear_pressure_profile_layered_harmonic():
    # columns of different permeability: constant flux through resistances
    # in series, p piecewise linear (harmonic two-point transmissibility)
    k = np.array([10.0, 300.0, 45.0, 2000.0, 80.0, 5.0])
    c = _linear_profile_case(k)
    a = bogen.assemble(c)
    dx = np.linalg.solve(_dense(a), a["b"])
    p = (c.x[0::3] + dx[0::3])[:6]
    h = c.dx
    # resistance (per unit area and mobility, up to a common factor) from the
    # left face to each cell centre
    res_to_centre = np.cumsum(np.concatenate([[h / 2 / k[0]], h / 2 / k[:-1] + h / 2 / k[1:]]))
    total = res_to_centre[-1] + h / 2 / k[-1]
    exact = 3500.0 - (3500.0 - 2500.0) * res_to_centre / total
    assert np.abs(p - exact).max() <= 1e-9 * 3500


def test_stone2_endpoint_identities():
    fl = default_fluid()
    swc = fl.swc
    for sw in [0.1, 0.2, 0.35, 0.6, 0.85]:
        # no gas: k_ro reduces to the oil-water curve k_row(Sw)
        krow = max(0.0, (1 - sw - fl.sorw) / (1 - swc - fl.sorw)) ** 2
        assert bogen.relperm(fl, sw, 0.0)[1] == pytest.approx(krow, abs=1e-15)
    for sg in [0.0, 0.05, 0.3, 0.6]:
        # connate water: k_ro reduces to the gas-oil curve k_rog(Sg)
        krog = max(0.0, (1 - sg - swc - fl.sorg) / (1 - swc - fl.sorg - fl.sgc)) ** 2
        assert bogen.relperm(fl, swc, sg)[1] == pytest.approx(krog, abs=1e-15)


def test_peaceman_equivalent_radius_square_cell():
    # isotropic square cell: r_o = 0.28 sqrt(2) dx / 2 ~= 0.198 dx
    dx, dz, k, rw = 100.0, 20.0, 150.0, 0.25
    ro = 0.14 * np.sqrt(2.0) * dx
    assert ro / dx == pytest.approx(0.198, abs=5e-4)
    wi = bogen.lib().bg_peaceman_wi(k, k, dx, dx, dz, rw, 0.0)
    assert wi == pytest.approx(0.001127 * 2 * np.pi * k * dz / np.log(ro / rw), rel=1e-14)


def _mobilities(fl, sw, sg):
    # at p = pref every formation volume factor is its reference value
    krw, kro, krg = bogen.relperm(fl, sw, sg)
    return krw / (fl.muw * fl.bw0), kro / (fl.muo * fl.bo0), krg / (fl.mug * fl.bg0), (krw, kro, krg)


@pytest.mark.parametrize("high", [0, 1])
def test_flux_is_upwinded_by_phase_potential(high):
    # two cells side by side, no gravity, x = x^n (no accumulation): each
    # phase flows with the mobility of the cell of higher potential, so cell 0
    # gets R = -T lambda_up (p_1 - p_0) per component (gas: dissolved plus free)
    fl = incompressible_fluid()
    c = bogen.uniform_case(2, 1, 1, fluid=fl)
    sat = [(0.6, 0.05), (0.2, 0.15)]
    p = [3000.0, 3000.0]
    p[high] = 3100.0
    c.x = np.array([p[0], *sat[0], p[1], *sat[1]])
    c.xn = c.x.copy()
    R = bogen.assemble(c, jacobian=False)["R"]
    T = 0.001127 * (c.dy * c.dz) * 100.0 / c.dx  # k = 100 mD in both cells
    lw, lo, lg, _ = _mobilities(fl, *sat[high])
    R0 = -T * (p[1] - p[0]) * np.array([lo, lw, fl.rs0 * lo + lg])
    assert np.allclose(R[0:3], R0, rtol=1e-12) and np.allclose(R[3:6], -R0, rtol=1e-12)


@pytest.mark.parametrize("kind", [0, 1])
def test_well_rates_closed_form(kind):
    # one cell at p = pref with one well (reference depth at the cell): R = -Q
    # with Q = WI lambda (p_bhp - p); the water injector uses the total
    # mobility over B_w, a producer each phase's own (gas: Rs lambda_o + lambda_g)
    fl = default_fluid()
    bhp = 3500.0 if kind == 0 else 2500.0
    c = bogen.uniform_case(1, 1, 1, p=3000.0, sw=0.3, sg=0.1, fluid=fl,
                           wells=[Well(kind, bhp, np.array([0], np.int32))])
    R = bogen.assemble(c, jacobian=False)["R"]
    wi = bogen.well_index(c, 0)
    lw, lo, lg, (krw, kro, krg) = _mobilities(fl, 0.3, 0.1)
    if kind == 0:
        q = np.array([0.0, (krw / fl.muw + kro / fl.muo + krg / fl.mug) / fl.bw0, 0.0])
    else:
        q = np.array([lo, lw, fl.rs0 * lo + lg])
    assert np.allclose(R, -wi * q * (bhp - 3000.0), rtol=1e-12, atol=0)


def test_oil_column_in_hydrostatic_equilibrium_has_no_oil_flow():
    # constant oil density rho_o and p = p_top + rho_o (D - D_top) / 144 make
    # every vertical oil potential difference vanish (Phi = p - rho g D / 144);
    # water and gas are lighter or heavier and still flow
    fl = incompressible_fluid(gravity=1.0)
    c = bogen.uniform_case(1, 1, 6, fluid=fl)
    rho_o = (fl.rhoo_sc * 5.615 + fl.rs0 * 1000.0 * fl.rhog_sc) / (5.615 * fl.bo0)
    c.x[0::3] = 3000.0 + rho_o * (c.depth - c.depth[0]) / 144.0
    c.xn = c.x.copy()
    R = bogen.assemble(c, jacobian=False)["R"]
    assert np.abs(R[1::3]).max() > 1e-3
    # against the oil flux one layer's gravity head would drive (rounding of
    # p ~ 3000 psi leaves about 1e-13 of it)
    _, lo, _, _ = _mobilities(fl, 0.2, 0.05)
    head_flux = 0.001127 * (c.dx * c.dy) * 100.0 / c.dz * lo * rho_o * c.dz / 144.0
    assert np.abs(R[0::3]).max() <= 1e-11 * head_flux


def test_tiny_case_is_seeded_and_nonsingular():
    a1 = bogen.assemble(bogen.tiny_case(0))
    a2 = bogen.assemble(bogen.tiny_case(0))
    assert np.array_equal(a1["val"], a2["val"]) and np.array_equal(a1["b"], a2["b"])
    a3 = bogen.assemble(bogen.tiny_case(1))
    assert not np.array_equal(a1["b"], a3["b"])
    assert np.all(np.isfinite(a1["val"]))


def test_learned_case_recipe():
    from bogen import learned as L
    c = L.learned_case(3, 32, 32, 16)
    c2 = L.learned_case(3, 32, 32, 16)
    assert np.array_equal(c.kx, c2.kx) and np.array_equal(c.x, c2.x)  # seeded
    inj, prod = c.wells
    assert inj.kind == 0 and prod.kind == 1 and inj.cells.size == 16 and prod.cells.size == 16
    ci, cp = int(inj.cells[0]), int(prod.cells[0])
    assert np.hypot(ci % 32 - cp % 32, ci // 32 - cp // 32) >= 16
    assert 3500 <= inj.bhp <= 4500 and 1500 <= prod.bhp <= 2500
    assert np.all((c.x[1::3] >= 0.1 - 1e-12) & (c.x[1::3] <= 0.85 + 1e-12))
    assert np.allclose(c.kz, 0.1 * c.kx)
    f = L.features(c)
    assert f.shape == (c.N, 16) and f.dtype == np.float32 and np.all(f[:, 6:] == 0)
    # well features only on perforated cells, signed by well type
    wells = np.zeros(c.N, bool)
    wells[inj.cells] = wells[prod.cells] = True
    assert np.all(f[~wells, 4] == 0) and np.all(f[inj.cells, 4] > 0) and np.all(f[prod.cells, 4] < 0)
    np.testing.assert_allclose(f[inj.cells, 5], (inj.bhp - c.x[0::3][inj.cells]) / 1000.0, rtol=1e-6)
    dx = np.arange(3 * c.N, dtype=np.float64)
    t = L.targets(dx)
    np.testing.assert_allclose(t[:, 0] * L.TARGET_SCALE[0], dx[0::3], rtol=1e-6)
    np.testing.assert_allclose(t[:, 2] * L.TARGET_SCALE[2], dx[2::3], rtol=1e-6)
    assert np.all(t[:, 3] == 0)


# ---------------------------------------------------------------- dual porosity
def test_dual_pattern_shape():
    from bogen import dual as D
    nx, ny, nz = 4, 3, 2
    N = nx * ny * nz
    rp, col = D.dual_pattern(nx, ny, nz)
    rp7, col7 = bogen.pattern(nx, ny, nz)
    assert rp.size == 2 * N + 1 and col.size == col7.size + 3 * N
    for c in range(N):
        row = list(col[rp[c]:rp[c + 1]])
        assert row == list(col7[rp7[c]:rp7[c + 1]]) + [N + c]
        assert sorted(col[rp[N + c]:rp[N + c + 1]]) == [c, N + c]


def test_dual_transfer_closed_form():
    # one cell, x = x^n, no wells: only the Warren-Root transfer remains,
    # tau = 0.001127 sigma k_m V lambda_up (Phi_f - Phi_m) out of the fracture
    # node (upstream: the node of higher pressure, here the fracture)
    from bogen import dual as D
    fl = incompressible_fluid()
    one = lambda v: np.array([float(v)])
    xf, xm = [3100.0, 0.5, 0.05], [3000.0, 0.2, 0.1]
    x = np.array(xf + xm)
    c = D.DualCase(1, 1, 1, 100.0, 100.0, 20.0, one(500), one(500), one(50), one(50), one(0.04), one(0.14),
                   one(8000.0), x, x.copy(), 1.0, sigma=0.1, wells=[], fluid=fl)
    R = D.assemble_dual(c)["R"]
    lw, lo, lg, _ = _mobilities(fl, xf[1], xf[2])
    tau = 0.001127 * 0.1 * 50.0 * (100.0 * 100.0 * 20.0) * (xf[0] - xm[0]) * np.array([lo, lw, fl.rs0 * lo + lg])
    assert np.allclose(R[0:3], tau, rtol=1e-12) and np.allclose(R[3:6], -tau, rtol=1e-12)


def test_dual_mass_balance_and_transfer_cancel():
    # summed over both continua, fluxes and the fracture-matrix transfer cancel:
    # sum R = accumulation of all 2N nodes (no wells)
    from bogen import dual as D
    c = D.dual_case(1, 6, 4, 3)
    c.wells = []
    rng = np.random.default_rng(2)
    N = c.N
    c.x = c.xn * rng.uniform(0.97, 1.03, 6 * N)
    a = D.assemble_dual(c)
    V = c.dx * c.dy * c.dz
    acc = np.zeros(3)
    for node in range(2 * N):
        phi = c.phif[node] if node < N else c.phim[node - N]
        for comp in range(3):
            m1 = bogen.cell_mass(c.fluid, phi, *c.x[3 * node:3 * node + 3], comp)
            m0 = bogen.cell_mass(c.fluid, phi, *c.xn[3 * node:3 * node + 3], comp)
            acc[comp] += V / (5.615 * c.dt) * (m1 - m0)
    tot = a["R"].reshape(2 * N, 3).sum(axis=0)
    assert np.allclose(tot, acc, rtol=1e-10, atol=1e-9 * np.abs(a["R"]).max())
    # the transfer moves fluid between the continua: per cell, the matrix
    # node's residual is its accumulation minus the inflow from its fracture
    assert np.abs(a["R"][3 * N:]).max() > 0


def test_dual_without_transfer_is_single_porosity_plus_storage():
    # shape factor 0: the fracture rows equal the single-porosity assembly of
    # the fracture continuum, and each matrix row holds only its accumulation block
    from bogen import dual as D
    c = D.dual_case(3, 6, 4, 3, shape_factor=0.0)
    N = c.N
    a = D.assemble_dual(c)
    sc = bogen.Case(c.nx, c.ny, c.nz, c.dx, c.dy, c.dz, c.kx, c.ky, c.kz, c.phif, c.depth, c.x[:3 * N].copy(),
                    c.xn[:3 * N].copy(), c.dt, c.wells, c.fluid)
    s = bogen.assemble(sc)
    rp, col = a["rowptr"], a["col"]
    for i in range(N):
        blocks = {int(col[e]): a["val"][e] for e in range(rp[i], rp[i + 1])}
        for e in range(s["rowptr"][i], s["rowptr"][i + 1]):
            np.testing.assert_array_equal(blocks[int(s["col"][e])], s["val"][e])
        assert np.all(blocks[N + i] == 0.0)
        mblocks = {int(col[e]): a["val"][e] for e in range(rp[N + i], rp[N + i + 1])}
        assert np.all(mblocks[i] == 0.0)
    np.testing.assert_array_equal(a["R"][:3 * N], s["R"])


def test_ensemble_recipe():
    # 256 seeded realisations of uneven size: nx, ny in [32, 96] (nx even for
    # the red-black layout), nz in [8, 24], sigma in [0.5, 2], and the total
    # unknown count inside the 38M-42M window
    s1, s2 = bogen.ensemble_specs(), bogen.ensemble_specs()
    assert s1 == s2 and len(s1) == 256
    d = np.array([sp["dims"] for sp in s1])
    assert np.all(d[:, 0] % 2 == 0)
    assert d[:, 0].min() >= 32 and d[:, 0].max() <= 96 and d[:, 1].min() >= 32 and d[:, 1].max() <= 96
    assert d[:, 2].min() >= 8 and d[:, 2].max() <= 24
    assert 38e6 <= 3 * int(np.prod(d, axis=1).sum()) <= 42e6
    assert all(0.5 <= sp["sigma"] <= 2.0 for sp in s1)
    assert len({sp["seed"] for sp in s1}) == 256
    # the sizes really are uneven
    cells = np.prod(d, axis=1)
    assert cells.max() > 5 * cells.min()


def test_waterflood_recipe():
    # the bench's Jacobian recipe at a reduced size: ln k_h = 4 + 1.5 g with g
    # of zero mean and unit variance, correlated over ~16 cells in x and ~2
    # layers in z (Gaussian filter of std s: lag-1 correlation exp(-1/(4 s^2)),
    # 0.999 and 0.94); k_v = 0.1 k_h; a water front around the four corner
    # injectors that grows with the day; BHP wells on whole columns
    nx, ny, nz = 64, 64, 16
    c0 = bogen.waterflood_case(nx, ny, nz, seed=42, day=0)
    c9 = bogen.waterflood_case(nx, ny, nz, seed=42, day=9)
    L = np.log(c0.kx).reshape(nz, ny, nx)
    assert abs(L.mean() - 4.0) < 1e-9 and abs(L.std() - 1.5) < 1e-9
    lag = lambda a, b: np.corrcoef(a.ravel(), b.ravel())[0, 1]
    assert lag(L[:, :, :-1], L[:, :, 1:]) > 0.99
    assert 0.85 < lag(L[:-1], L[1:]) < 0.97
    assert np.array_equal(c0.kx, c0.ky) and np.allclose(c0.kz, 0.1 * c0.kx, rtol=1e-15)
    assert np.array_equal(c0.kx, c9.kx)  # the day moves the front only
    sw0, sw9 = c0.x[1::3], c9.x[1::3]
    assert sw0.min() >= 0.1 and sw0.max() <= 0.85
    assert sw9.mean() > sw0.mean()
    assert np.all(c0.x[2::3] == 0.05) and np.array_equal(c0.x, c0.xn)
    assert np.allclose(c0.x[0::3], 3000.0 + 0.35 * (c0.depth - c0.depth.min() + 10.0))
    inj = [w for w in c0.wells if w.kind == 0]
    prod = [w for w in c0.wells if w.kind == 1]
    assert len(inj) == 4 and len(prod) == 1
    assert all(w.bhp == 4000.0 and w.cells.size == nz for w in inj) and prod[0].bhp == 2000.0
    corners = {(int(w.cells[0]) % nx, int(w.cells[0]) // nx) for w in inj}
    assert corners == {(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1)}
    assert int(prod[0].cells[0]) == nx // 2 + nx * (ny // 2)
    assert not np.array_equal(c0.kx, bogen.waterflood_case(nx, ny, nz, seed=43).kx)


def test_dual_porosity_recipe():
    # fracture permeability 10 k_m with ln k_m = 4 + sigma g (sigma in
    # [0.5, 2]), porosities 0.04 / 0.14, shape factor 0.1 ft^-2; the matrix
    # lags the fractures: p_m <= p_f, Sw_m = 0.1 + 0.5 (Sw_f - 0.1); wells on
    # the fracture columns at (0, 0) and (nx-1, ny-1)
    from bogen import dual as D
    nx, ny, nz = 12, 10, 4
    c = D.dual_case(5, nx, ny, nz)
    N = nx * ny * nz
    Lm = np.log(c.km)
    assert abs(Lm.mean() - 4.0) < 1e-9 and 0.5 - 1e-9 <= Lm.std() <= 2.0 + 1e-9
    assert np.allclose(c.kx, 10.0 * c.km, rtol=1e-15) and np.array_equal(c.kx, c.kz)
    assert np.all(c.phif == 0.04) and np.all(c.phim == 0.14) and c.sigma == 0.1
    xf, xm = c.x[:3 * N], c.x[3 * N:]
    assert np.all(xm[0::3] <= xf[0::3])
    assert np.allclose(xm[1::3], 0.1 + 0.5 * (xf[1::3] - 0.1), rtol=0, atol=1e-15)
    assert np.all(xf[2::3] == 0.05) and np.all(xm[2::3] == 0.05) and np.array_equal(c.x, c.xn)
    assert xf[1::3].min() >= 0.1 and xf[1::3].max() <= 0.85
    inj, prod = c.wells
    assert (inj.kind, inj.bhp, int(inj.cells[0])) == (0, 4000.0, 0)
    assert (prod.kind, prod.bhp, int(prod.cells[0])) == (1, 2000.0, nx - 1 + nx * (ny - 1))
    assert inj.cells.size == prod.cells.size == nz and np.all(inj.cells < N)
