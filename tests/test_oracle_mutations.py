"""Planted mistakes: each case compiles a copy of oracle.cpp with one
plausible error (a flipped sign, a transposed index, a wrong update) and runs
the pin that should catch it against that copy; the pin must fail.  The
unaltered source, compiled the same way, must pass the same pins.  This
checks that the pins constrain the oracle rather than restate it."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.cpp")

# (what is wrong, exact source text, altered text, pin file, pin tests that must fail)
P = "test_oracle_pins.py"
L = "test_oracle_learned_pins.py"
MUTATIONS = [
    ("BSR SpMV reads the block transposed",
     "s += val[(size_t)e * bs * bs + bs * r + c] * x[(size_t)col[e] * bs + c];",
     "s += val[(size_t)e * bs * bs + bs * c + r] * x[(size_t)col[e] * bs + c];",
     P, "test_spmv_matches_dense_product"),
    ("Quasi-IMPES weight of the water row has the wrong sign",
     "{1.0, -D[1] / D[4], -D[2] / D[8]}", "{1.0, D[1] / D[4], -D[2] / D[8]}",
     P, "test_qi_operator_multiplied_back_gives_A"),
    ("Exact local decoupling takes a column of A_ii^{-1} instead of row 0",
     "Dt[3 * r + c] = D[3 * c + r];", "Dt[3 * r + c] = D[3 * r + c];",
     P, "test_flooded_injector_cells_take_exact_local_decoupling"),
    ("ILU(0) elimination adds instead of subtracts",
     "lu[(size_t)f * b2 + t] -= prod[t];", "lu[(size_t)f * b2 + t] += prod[t];",
     P, "test_ilu0_defining_property"),
    ("ILU(0) backward substitution adds the upper blocks",
     "s[rr] -= lu[(size_t)e * b2 + bs * rr + c] * z[k * bs + c];",
     "s[rr] += lu[(size_t)e * b2 + bs * rr + c] * z[k * bs + c];",
     P, "test_ilu0_exact_on_block_tridiagonal_column"),
    ("Permutation inverted the wrong way",
     "inv[perm[i]] = i;", "inv[i] = perm[i];",
     P, "test_permute_matches_dense_permutation"),
    ("Dense LU forgets the row interchanges in the solve",
     "for (int k = 0; k < n; ++k) std::swap(y[k], y[piv[k]]);", "",
     P, "test_dense_solve_matches_lapack"),
    ("Relative residual adds A x instead of subtracting it",
     "s.add(-val[(size_t)e * bs * bs + bs * r + c] * x[(size_t)col[e] * bs + c]);",
     "s.add(val[(size_t)e * bs * bs + bs * r + c] * x[(size_t)col[e] * bs + c]);",
     P, "test_rel_residual_matches_numpy"),
    ("Galerkin coarse operator transposed",
     "rows[f.agg[i]][f.agg[f.A.col[e]]] += f.A.val[e];", "rows[f.agg[f.A.col[e]]][f.agg[i]] += f.A.val[e];",
     P, "test_amg_galerkin_on_a_nonsymmetric_matrix"),
    ("Restriction keeps one residual per aggregate instead of the sum",
     "fc[L.agg[i]] += r;", "fc[L.agg[i]] = r;",
     P, "test_amg_two_level_without_smoothing_is_scaled_coarse_correction"),
    ("Over-correction factor dropped",
     "x[i] += prm.overcorr * xc[L.agg[i]];", "x[i] += xc[L.agg[i]];",
     P, "test_amg_two_level_without_smoothing_is_scaled_coarse_correction"),
    ("Jacobi sweep undamped",
     "xn[i] = x[i] + prm.omega * s / d;", "xn[i] = x[i] + s / d;",
     P, "test_amg_two_level_jacobi_cycle_closed_form"),
    ("Post-smoothing repeats the red-black order",
     "gs_half(L, pre ? 0 : 1, f, x);\n        gs_half(L, pre ? 1 : 0, f, x);",
     "gs_half(L, 0, f, x);\n        gs_half(L, 1, f, x);",
     P, "test_amg_two_level_gauss_seidel_cycle_closed_form or test_amg_symmetric_vcycle_is_symmetric_operator"),
    ("CPR places the pressure correction on the water unknown",
     "for (int64_t i = 0; i < nb; ++i) x[3 * i] += ep[i];",
     "for (int64_t i = 0; i < nb; ++i) x[3 * i + 1] += ep[i];",
     P, "test_cpr_stages_compose_as_alg2"),
    ("CPR decouples the input with the wrong gas entry",
     "w[3 * i + 2] * v[3 * i + 2];", "w[3 * i + 2] * v[3 * i + 1];",
     P, "test_cpr_stages_compose_as_alg2"),
    ("GMRES Givens rotation with the wrong sine",
     "sn[j] = c / d;", "sn[j] = -c / d;",
     P, "test_gmres_matches_lapack_on_small_black_oil"),
    ("GMRES Gram-Schmidt adds the projection",
     "for (int64_t t = 0; t < n; ++t) w[t] -= h * V[i][t];",
     "for (int64_t t = 0; t < n; ++t) w[t] += h * V[i][t];",
     P, "test_gmres_matches_lapack_on_small_black_oil"),
    ("BiCGSTAB update subtracts the minimal-residual step",
     "x[i] += alpha * ph[i] + omega * sh[i];", "x[i] += alpha * ph[i] - omega * sh[i];",
     P, "test_bicgstab_matches_lapack_on_small_black_oil"),
    ("BiCGSTAB search direction without the omega term",
     "p[i] = r[i] + beta * (p[i] - omega * v[i]);", "p[i] = r[i] + beta * p[i];",
     P, "test_bicgstab_matches_lapack_on_small_black_oil"),
    ("Learned coarse operator uses zc of the row cell twice",
     "zc[c] * App.val[e] * zc[App.col[e]];", "zc[c] * App.val[e] * zc[c];",
     L, "test_galerkin_orthogonality"),
]


# The same for the oracle's Python modules: (what is wrong, module, exact
# source text, altered text, pin file, pin tests that must fail)
C = "test_oracle_cnn_pins.py"
N = "test_oracle_newton_pins.py"
WP = "test_oracle_wells_pins.py"
OW = "test_oracle_oilwater_pins.py"
PY_MUTATIONS = [
    ("Convolution instead of correlation (taps mirrored)",
     "cnn.py", "y += _window(xp, dx, dy, dz, nz, ny, nx) @ w[t].T", "y += _window(xp, dx, dy, dz, nz, ny, nx) @ w[26 - t].T",
     C, "test_single_channel_matches_scipy_correlate or test_brute_force_small"),
    ("Data gradient scatters through the unmirrored offset",
     "cnn.py", "_window(dxp, dx, dyy, dz, nz, ny, nx)[...] += dy @ w[t]",
     "_window(dxp, -dx, -dyy, -dz, nz, ny, nx)[...] += dy @ w[t]",
     C, "test_backward_data_is_adjoint"),
    ("Bias gradient averaged instead of summed",
     "cnn.py", "return dw, d2.sum(axis=0)", "return dw, d2.mean(axis=0)",
     C, "test_backward_weights_is_adjoint or test_gradient_matches_finite_differences"),
    ("Residual block adds the wrong activation",
     "cnn.py", "y = y + acts[l - 1]", "y = y + acts[l]",
     C, "test_zero_second_conv_makes_block_pass_through"),
    ("Backward pass drops the skip connection",
     "cnn.py", "g = g + skip  #", "g = g  #",
     C, "test_gradient_matches_finite_differences"),
    ("Adam without bias correction",
     "cnn.py", "mh = m / (1.0 - b1 ** t)", "mh = m",
     C, "test_adam_first_steps_closed_form"),
    ("Newton step damped by one half (linear, not quadratic, convergence)",
     "newton.py", "x = x + dx", "x = x + 0.5 * dx",
     N, "test_exact_newton_converges_quadratically"),
    ("Linear residual of the Newton step with the wrong sign",
     "newton.py", "r = b - matvec(A, dx)", "r = b + matvec(A, dx)",
     N, "test_forcing_terms_reach_the_same_solution_with_fewer_linear_iterations"),
    ("First forcing term with numerator and denominator swapped",
     "newton.py", "return float(np.linalg.norm(b_new - r)) / nb_old",
     "return nb_old / float(np.linalg.norm(b_new - r))",
     N, "test_forcing_terms_by_hand_on_one_unknown"),
    ("First forcing term with the old residual in place of the linear residual",
     "newton.py", "return float(np.linalg.norm(b_new - r)) / nb_old",
     "return float(np.linalg.norm(b_new + r)) / nb_old",
     N, "test_forcing_terms_by_hand_on_one_unknown"),
    ("Second forcing term with numerator and denominator swapped",
     "newton.py", "return abs(float(np.linalg.norm(b_new)) - float(np.linalg.norm(r))) / nb_old",
     "return nb_old / abs(float(np.linalg.norm(b_new)) - float(np.linalg.norm(r)))",
     N, "test_forcing_terms_by_hand_on_one_unknown"),
    ("Second forcing term without the absolute value",
     "newton.py", "return abs(float(np.linalg.norm(b_new)) - float(np.linalg.norm(r))) / nb_old",
     "return (float(np.linalg.norm(b_new)) - float(np.linalg.norm(r))) / nb_old",
     N, "test_forcing_terms_by_hand_on_one_unknown"),
    ("Third forcing term with the ratio inverted",
     "newton.py", "return gamma * (float(np.linalg.norm(b_new)) / nb_old) ** beta",
     "return gamma * (nb_old / float(np.linalg.norm(b_new))) ** beta",
     N, "test_forcing_terms_by_hand_on_one_unknown"),
    ("Third forcing term without gamma",
     "newton.py", "return gamma * (float(np.linalg.norm(b_new)) / nb_old) ** beta",
     "return (float(np.linalg.norm(b_new)) / nb_old) ** beta",
     N, "test_forcing_terms_by_hand_on_one_unknown"),
    ("Well column entries placed in the well's row of the cell block",
     "bordered.py", "blk[:, 0] = apw[e]", "blk[0, :] = apw[e]",
     WP, "test_bordered_matrix_is_the_jacobian_of_the_full_residual"),
    ("Well diagonal block without A_ww",
     "bordered.py", "vals.append(np.diag([aww[w], 1.0, 1.0]))", "vals.append(np.diag([1.0, 1.0, 1.0]))",
     WP, "test_bordered_matrix_is_the_jacobian_of_the_full_residual"),
    ("Well unknown embedded in the wrong slot of its block row",
     "bordered.py", "out[3 * N::3] = v[3 * N:]", "out[3 * N + 1::3] = v[3 * N:]",
     WP, "test_bordered_solve_matches_dense_lu"),
    ("ABF scaling applied on the right (A D^{-1})",
     "__init__.py", "val[e] = Dinv @ A.val[e]", "val[e] = A.val[e] @ Dinv",
     OW, "test_abf_decoupling_identities"),
    ("Padded two-phase matrix without the third unknown's unit diagonal",
     "__init__.py", "val[e, 2, 2] = 1.0", "val[e, 2, 2] = 0.0",
     OW, "test_two_phase_reference_solutions_match_dense_lu"),
    ("Safeguard clips at theta_min only",
     "newton.py", "theta = min(max(forcing_term(forcing, b_new, nb_old, r, gamma, beta), theta_min), theta_max)",
     "theta = max(forcing_term(forcing, b_new, nb_old, r, gamma, beta), theta_min)",
     N, "test_forcing_term_safeguards"),
]


# The seeded Jacobian generator the oracle's inputs come from, against its
# physics pins: (what is wrong, exact source text, altered text, pin tests)
G = "test_generator_pins.py"
GEN_SRC = os.path.join(ROOT, "bogen", "assembly.cpp")
GEN_MUTATIONS = [
    ("Quotient rule with the wrong sign",
     "r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);", "r.d[i] = (a.d[i] * b.v + a.v * b.d[i]) / (b.v * b.v);",
     "test_exact_jacobian_matches_central_differences"),
    ("Arithmetic instead of harmonic face permeability",
     "    return kDarcy * area * 2.0 / (h / k1 + h / k2);\n  };",
     "    return kDarcy * area * (k1 + k2) / (2.0 * h);\n  };",
     "test_face_transmissibility_is_harmonic or test_linear_pressure_profile_layered_harmonic"),
    ("Flux added to the neighbour with the wrong sign",
     "R[3 * b + comp] += F[comp]->v;", "R[3 * b + comp] -= F[comp]->v;",
     "test_component_mass_balance"),
    ("Upwinding takes the downstream cell",
     "if (d.v > 0) return lift(qb, 3);\n    if (d.v < 0) return lift(qa, 0);",
     "if (d.v > 0) return lift(qa, 0);\n    if (d.v < 0) return lift(qb, 3);",
     "test_flux_is_upwinded_by_phase_potential"),
    ("Accumulation adds the previous mass",
     "R[3 * c + comp] += s * (m[comp]->v - mn);", "R[3 * c + comp] += s * (m[comp]->v + mn);",
     "test_component_mass_balance"),
    ("Water injector with the water mobility instead of the total",
     "qw = WI * C.lt_res_w * dpw;", "qw = WI * C.lw * dpw;",
     "test_well_rates_closed_form"),
    ("Gravity term of the oil potential with the wrong sign",
     "Dual<6> dphi_o = (pb - pa) - 0.5 *", "Dual<6> dphi_o = (pb - pa) + 0.5 *",
     "test_oil_column_in_hydrostatic_equilibrium_has_no_oil_flow"),
    ("Stone II without the gas term",
     "(krog / krocw + krg) - krw - krg));", "(krog / krocw + krg) - krw));",
     "test_stone2_endpoint_identities"),
    ("Peaceman radius with the wrong constant",
     "const double ro = 0.28 *", "const double ro = 0.14 *",
     "test_peaceman_equivalent_radius_square_cell"),
    ("Pattern lists the wrong y neighbour",
     "if (j < ny - 1) col[e++] = (int32_t)(c + nx);", "if (j < ny - 1) col[e++] = (int32_t)(c + ny);",
     "test_pattern_is_seven_point_sorted"),
    ("Dual-porosity transfer without the bulk volume",
     "kDarcy * sigma * km[c] * V, R);", "kDarcy * sigma * km[c], R);",
     "test_dual_transfer_closed_form"),
    ("Well column of the border with the wrong sign",
     "apw[3 * e + comp] = -Q[comp]->d[3];", "apw[3 * e + comp] = Q[comp]->d[3];",
     "test_border_matches_central_differences"),
    ("Liquid-rate control without the water rate",
     "const Dual<4> qc = ctrl[w] == 1 ? qw : ctrl[w] == 2 ? qo : qo + qw;",
     "const Dual<4> qc = ctrl[w] == 1 ? qw : ctrl[w] == 2 ? qo : qo;",
     "test_newton_meets_the_rate_targets"),
    ("Dirichlet face transmissibility over a whole cell",
     "kx[c] / (0.5 * g->dx);", "kx[c] / g->dx;",
     "test_linear_pressure_profile_homogeneous"),
]


def _compile(tmp_path, name, text):
    src = tmp_path / f"{name}.cpp"
    src.write_text(text)
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-pthread", "-shared", "-fPIC", str(src), "-o", str(so)])
    return str(so)


def _run_pins(lib, files, tests):
    env = dict(os.environ, BO_ORACLE_LIB=lib)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
           *[os.path.join(ROOT, "tests", f) for f in sorted(set(files))], "-k", tests]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True)


@pytest.fixture(scope="module")
def original_lib(tmp_path_factory):
    return _compile(tmp_path_factory.mktemp("oracle"), "original", open(SRC).read())


def test_unaltered_oracle_passes_the_pins(original_lib):
    lib = original_lib
    r = _run_pins(lib, [m[3] for m in MUTATIONS], " or ".join(m[4] for m in MUTATIONS))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("what,orig,bad,pinfile,pin", MUTATIONS, ids=[f"m{i:02d}" for i in range(len(MUTATIONS))])
def test_planted_mistake_is_caught(tmp_path, what, orig, bad, pinfile, pin):
    text = open(SRC).read()
    assert text.count(orig) == 1, f"mutation site not unique or missing: {orig}"
    lib = _compile(tmp_path, "mutant", text.replace(orig, bad))
    r = _run_pins(lib, [pinfile], pin)
    assert r.returncode != 0, f"{what}: the pin {pin} still passed"


def _oracle_copy(tmp_path, module, orig, bad):
    import shutil
    dst = tmp_path / "pkg" / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), dst, ignore=shutil.ignore_patterns("__pycache__", "*.so"))
    text = (dst / module).read_text()
    assert text.count(orig) == 1, f"mutation site not unique or missing: {orig}"
    (dst / module).write_text(text.replace(orig, bad))
    return str(tmp_path / "pkg")


@pytest.mark.parametrize("what,module,orig,bad,pinfile,pin", PY_MUTATIONS,
                         ids=[f"py{i:02d}" for i in range(len(PY_MUTATIONS))])
def test_planted_mistake_in_python_oracle_is_caught(tmp_path, original_lib, what, module, orig, bad, pinfile, pin):
    lib = original_lib
    pkg = _oracle_copy(tmp_path, module, orig, orig)
    env = dict(os.environ, BO_ORACLE_LIB=lib, BO_ORACLE_PATH=pkg)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
           os.path.join(ROOT, "tests", pinfile), "-k", pin]
    # the unaltered copy passes, so a failure below is the planted mistake's
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout[-2000:]
    import shutil
    shutil.rmtree(os.path.join(pkg, "oracle"))
    pkg = _oracle_copy(tmp_path, module, orig, bad)
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True)
    assert r.returncode != 0, f"{what}: the pin {pin} still passed"


@pytest.fixture(scope="module")
def original_gen_lib(tmp_path_factory):
    return _compile(tmp_path_factory.mktemp("bogen"), "bogen_original", open(GEN_SRC).read())


def _run_gen_pins(lib, tests):
    env = dict(os.environ, BO_BOGEN_LIB=lib)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
           os.path.join(ROOT, "tests", G), os.path.join(ROOT, "tests", WP), "-k", tests]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True)


def test_unaltered_generator_passes_the_pins(original_gen_lib):
    r = _run_gen_pins(original_gen_lib, " or ".join(m[3] for m in GEN_MUTATIONS))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("what,orig,bad,pin", GEN_MUTATIONS, ids=[f"gen{i:02d}" for i in range(len(GEN_MUTATIONS))])
def test_planted_mistake_in_generator_is_caught(tmp_path, what, orig, bad, pin):
    text = open(GEN_SRC).read()
    assert text.count(orig) == 1, f"mutation site not unique or missing: {orig}"
    lib = _compile(tmp_path, "bogen_mutant", text.replace(orig, bad))
    r = _run_gen_pins(lib, pin)
    assert r.returncode != 0, f"{what}: the pin {pin} still passed"
