"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake, the kind a reader might miss: a dropped
term, a wrong sign, index, exponent or factor, a transposed operand, swapped
substeps. The oracle's pin tests (tests/test_oracle_*.py) then run against
it in a subprocess. A mistake counts as caught when some pin fails.

- A mistake in oracle/hc_oracle.c: the mutated copy is built into its own
  library in a temporary folder, and the pins load it through HC_ORACLE_LIB.
- A mistake in oracle/__init__.py, the host logic such as Algorithm 1's loop
  and its stopping rules: the pins run in a temporary copy of the tests, the
  oracle package and the input generators, with the mutated module.

The unchanged sources, run the same two ways, must pass every pin: that shows
the harness itself is sound. Everything runs on the CPU. The mistakes live
only in temporary copies."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hc_oracle.c")
HDR = os.path.join(ROOT, "oracle", "hc_oracle.h")
PY_SRC = os.path.join(ROOT, "oracle", "__init__.py")
PIN_TESTS = sorted(
    os.path.join("tests", f) for f in os.listdir(os.path.join(ROOT, "tests"))
    if f.startswith("test_oracle_") and f.endswith(".py"))

# (name, text in hc_oracle.c, replacement)
MUTANTS = [
    # transforms and Fourier variables
    ("dft_sign", "double ang = sign * 2.0 * M_PI * (double)jk / n;",
     "double ang = -sign * 2.0 * M_PI * (double)jk / n;"),
    ("fft_twiddle_sign", "double ang = sign * 2.0 * M_PI * (double)k / n;",
     "double ang = -sign * 2.0 * M_PI * (double)k / n;"),
    ("fft_butterfly_order", "a[s + k + half] = u - v;", "a[s + k + half] = v - u;"),
    ("xi_nyquist_negative", "return (l <= N / 2) ?", "return (l < N / 2) ?"),
    ("xi_deriv_nyquist_kept", "if (2 * l == N) return 0.0; /* R1 */", "if (0) return 0.0;"),
    ("gradient_sign",
     "t[q] = I * or_xi_deriv(coord(g, q, c), g->n[c], g->L[c]) * fh[q];",
     "t[q] = -I * or_xi_deriv(coord(g, q, c), g->n[c], g->L[c]) * fh[q];"),
    ("gradient_wrong_length",
     "t[q] = I * or_xi_deriv(coord(g, q, c), g->n[c], g->L[c]) * fh[q];",
     "t[q] = I * or_xi_deriv(coord(g, q, c), g->n[c], g->L[0]) * fh[q];"),
    # pressure operator
    ("K_drops_r", "m[(size_t)c * npts + p] * mv + r[p] * v[(size_t)c * npts + p];",
     "m[(size_t)c * npts + p] * mv;"),
    ("K_transposed_rank_one", "m[(size_t)c * npts + p] * mv + r[p]",
     "v[(size_t)c * npts + p] * mv + r[p]"),
    ("A_divergence_sign", "Ap[q] = -creal(div[q]);", "Ap[q] = creal(div[q]);"),
    # Not a mistake, so not listed: keeping +pi N / L at the Nyquist index of the
    # divergence. There i xi multiplies a self-conjugate coefficient, and the real part
    # of the inverse transform drops the result, as reading R1 states.
    ("A_divergence_wrong_axis",
     "div[q] += I * or_xi_deriv(coord(g, q, c), g->n[c], g->L[c]) * t[q];",
     "div[q] += I * or_xi_deriv(coord(g, q, 0), g->n[0], g->L[0]) * t[q];"),
    ("projection_wrong_mean", "s /= (double)npts;", "s /= (double)(npts - 1);"),
    ("projection_odd_axes_have_nyquist", "if (((e >> a) & 1) && (g->n[a] % 2)) ok = 0;",
     "if (0) ok = 0;"),
    ("projection_parity_of_one_axis",
     "        if ((e >> a) & 1) par += coord(g, q, a);\n      s += ",
     "        if ((e >> a) & 1) par += coord(g, q, 0);\n      s += "),
    ("fft_axis_stride", "for (int b = 0; b < ax; ++b) stride *= (size_t)g->n[b];",
     "for (int b = 0; b < ax && b < 1; ++b) stride *= (size_t)g->n[b];"),
    # preconditioner and CG
    ("precond_symbol_index", "s += xi[a] * kbar_at(kbar, a, b) * xi[b];",
     "s += xi[a] * kbar_at(kbar, a, a) * xi[b];"),
    ("kbar_index_table_xz_yz", "static const int idx[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};",
     "static const int idx[3][3] = {{0, 3, 5}, {3, 1, 4}, {5, 4, 2}};"),
    ("kbar_pairs_swapped", "pb[6] = {0, 1, 2, 1, 2, 2};", "pb[6] = {0, 1, 2, 1, 1, 2};"),
    ("kappa_fixed_dimension", "return sr / (double)npts + sm / (double)npts / (double)g->dim;",
     "return sr / (double)npts + sm / (double)npts / 2.0;"),
    ("dot_skips_last_entry", "for (size_t i = 0; i < n; ++i) s += a[i] * b[i];",
     "for (size_t i = 0; i + 1 < n; ++i) s += a[i] * b[i];"),
    ("kbar_offdiag_square", "s += m[(size_t)pa[e] * npts + q] * m[(size_t)pb[e] * npts + q];",
     "s += m[(size_t)pa[e] * npts + q] * m[(size_t)pa[e] * npts + q];"),
    ("kappa_no_dim_division", "return sr / (double)npts + sm / (double)npts / (double)g->dim;",
     "return sr / (double)npts + sm / (double)npts;"),
    ("precond_option_swapped", "if (prm->kappa > 0 || prm->precond != 1) {",
     "if (prm->kappa > 0 || prm->precond == 1) {"),
    ("cg_no_initial_projection",
     "or_project(g, x); /* initial guess into the complement of the null space (R2) */", ""),
    ("cg_absolute_stop", "while (rnorm > rtol * bnorm && it < maxit) {",
     "while (rnorm > rtol && it < maxit) {"),
    ("cg_beta_inverted", "double beta = rho_new / rho;", "double beta = rho / rho_new;"),
    ("cg_alpha_wrong_denominator", "const double dAd = dot(n, d, q);",
     "const double dAd = dot(n, d, d);"),
    # splitting substeps
    ("activation_exponent_sign", "double e = exp(c * c * g2 * dt);", "double e = exp(-c * c * g2 * dt);"),
    ("activation_gperp_sign", "double gperp[2] = {-g[1], g[0]};", "double gperp[2] = {g[1], g[0]};"),
    ("activation_norm_drops_z", "double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];",
     "double g2 = g[0] * g[0] + g[1] * g[1];"),
    ("activation_3d_drops_projection",
     "out[a] = mm[a] - g[a] * gm / g2 + g[a] * gm * e / g2;",
     "out[a] = mm[a] + g[a] * gm * e / g2;"),
    ("relaxation_exponent", "pow(b, 1.0 / (2.0 * (1.0 - gamma)))", "pow(b, 1.0 / (1.0 - gamma))"),
    ("relaxation_dt_factor", "- 2.0 * (1.0 - gamma) * dt;", "- (1.0 - gamma) * dt;"),
    ("relaxation_no_indicator", "double scale = (b >= 0) ?", "double scale = (1) ?"),
    ("relaxation_gamma_one_loose_compare", "if (gamma == 1.0) { /* m exp(-dt) */",
     "if (fabs(gamma - 1.0) < 0.3) { /* m exp(-dt) */"),
    ("relaxation_gamma_one_sign", "*= exp(-dt);\n      continue;", "*= exp(dt);\n      continue;"),
    ("diffusion_D_not_squared", "t[q] *= exp(-D * D * s * dt);", "t[q] *= exp(-D * s * dt);"),
    ("diffusion_drops_nyquist", "double x = or_xi(coord(g, q, a), g->n[a], g->L[a]);",
     "double x = or_xi_deriv(coord(g, q, a), g->n[a], g->L[a]);"),
    # loops that stop at two dimensions
    ("diffusion_wavenumber_2d_only", "      for (int a = 0; a < g->dim; ++a) {\n        double x = or_xi(",
     "      for (int a = 0; a < 2; ++a) {\n        double x = or_xi("),
    ("energy_grad_m_two_components",
     "  for (int c = 0; c < dim; ++c) {\n    or_gradient(g, m + (size_t)c * npts, gm);",
     "  for (int c = 0; c < 2; ++c) {\n    or_gradient(g, m + (size_t)c * npts, gm);"),
    ("energy_pointwise_two_components",
     "    for (int c = 0; c < dim; ++c) {\n      double gc = gp[(size_t)c * npts + q]",
     "    for (int c = 0; c < 2; ++c) {\n      double gc = gp[(size_t)c * npts + q]"),
    ("precond_symbol_two_axes",
     "    for (int a = 0; a < g->dim; ++a)\n      for (int b = 0; b < g->dim; ++b) s += xi[a]",
     "    for (int a = 0; a < 2; ++a)\n      for (int b = 0; b < 2; ++b) s += xi[a]"),
    ("gradient_two_components", "  for (int c = 0; c < g->dim && !rc; ++c) {\n    /* d f / d x_c",
     "  for (int c = 0; c < 2 && !rc; ++c) {\n    /* d f / d x_c"),
    # Algorithm 1's order
    ("step_relaxation_before_activation",
     "or_activation(dim, npts, m, grad, prm->c, prm->dt);\n    or_relaxation(dim, npts, m, prm->gamma, prm->dt);",
     "or_relaxation(dim, npts, m, prm->gamma, prm->dt);\n    or_activation(dim, npts, m, grad, prm->c, prm->dt);"),
    ("step_gradient_of_source", "  if (!rc) rc = or_gradient(g, p, grad);\n  if (!rc) {",
     "  if (!rc) rc = or_gradient(g, b, grad);\n  if (!rc) {"),
    ("step_no_source_projection",
     "or_project(g, b); /* solvability: S orthogonal to the null space (R2) */", ""),
    # energy
    ("energy_one_derivative_direction", "q < (size_t)dim * npts; ++q) e_diff", "q < npts; ++q) e_diff"),
    ("energy_flow_term_factor", "0.5 * c2 * e_r +", "c2 * e_r +"),
    ("energy_flow_uses_m_squared", "mg += mc * gc;", "mg += mc * mc;"),
    ("energy_gamma0_drops_log_term", "prm->gamma != 0.0 ? e_rel / (2.0 * prm->gamma) : e_rel",
     "prm->gamma != 0.0 ? e_rel / (2.0 * prm->gamma) : 0.0"),
    ("energy_gamma0_log_of_m_squared", "e_rel += 0.5 * log(m2);", "e_rel += log(m2);"),
    ("energy_gamma0_log_drops_zeros", "e_rel += 0.5 * log(m2);", "e_rel += m2 > 0 ? 0.5 * log(m2) : 0.0;"),
    ("energy_gamma_power", "e_rel += pow(m2, prm->gamma);", "e_rel += pow(m2, 2.0 * prm->gamma);"),
    # adjoint. Not listed, because they change nothing: dropping the projection of
    # lambda_p, a spectral divergence with no null-mode content; and dropping the final
    # projection of dL/dS, a sum of adjoint pressures that CG keeps in the complement.
    ("adjoint_relax_gamma_one", "if (gamma == 1.0) { *c1 = exp(-dt);", "if (gamma == 1.0) { *c1 = 1.0;"),
    ("adjoint_pressure_of_wrong_step", "const double* p = ps + n * (k + 1); /* solved with m^k */",
     "const double* p = ps + n * k;"),
    ("adjoint_divergence_sign", "lp[q] -= creal(ct[q]);", "lp[q] += creal(ct[q]);"),
    ("adjoint_dr_sign", "dr[q] -= gm[0] * gp[0]", "dr[q] += gm[0] * gp[0]"),
    ("adjoint_drops_dphi_term", " + 2.0 * c2 * dtt * dph * mg * gl * gv[c]);", ");"),
    ("adjoint_dphi1_series", "s += term / (k + 2);", "s += term / (k + 1);"),
    ("adjoint_dD2_missing_dt", "ct[q] *= -s2 * dtt * exp(-D2 * s2 * dtt);",
     "ct[q] *= -s2 * exp(-D2 * s2 * dtt);"),
    ("adjoint_relax_jacobian", "* pow(rho, e - 1.0); /* df/drho */", "* pow(rho, e); /* df/drho */"),
    ("adjoint_drops_symmetric_m_term", "-= gm[c] * mgp + gp[c] * mgm;", "-= gm[c] * mgp;"),
    ("adjoint_dc2_drops_dphi", "*dc2 += gl * mg * dtt * (ph + z * dph);", "*dc2 += gl * mg * dtt * ph;"),
    ("adjoint_lambda_drops_activation",
     "lam[(size_t)c * n + q] = la[c] + c2 * dtt * ph * gl * gv[c];", "lam[(size_t)c * n + q] = la[c];"),
    ("adjoint_factor_two", "2.0 * c2 * dtt * dph * mg * gl * gv[c]", "1.0 * c2 * dtt * dph * mg * gl * gv[c]"),
    ("adjoint_relax_unnormalised", "*c2 = (fp - sv) / n2;", "*c2 = (fp - sv);"),
    ("adjoint_relax_zero_branch", "if (n2 == 0) { *c1 = gamma > 1.0 ? 1.0 : 0.0; *c2 = 0; return; }",
     "if (n2 == 0) { *c1 = 1.0; *c2 = 0; return; }"),
    ("adjoint_relax_extinct_branch", "if (beta <= 0) { *c1 = 0; *c2 = 0; return; }",
     "if (beta <= 0) { *c1 = 1; *c2 = 0; return; }"),
    ("adjoint_dD2_sign", "ct[q] *= -s2 * dtt * exp(-D2 * s2 * dtt);", "ct[q] *= s2 * dtt * exp(-D2 * s2 * dtt);"),
    ("adjoint_skips_heat_transpose", "rc = or_diffusion(g, lb, prm->D, dtt);", "rc = 0;"),
    ("adjoint_m_dot_g_drops_z", "double mg = mv[0] * gv[0] + mv[1] * gv[1] + mv[2] * gv[2];",
     "double mg = mv[0] * gv[0] + mv[1] * gv[1];"),
    ("adjoint_lambda_g_swapped", "ph * (mg * la[c] + mv[c] * gl)", "ph * (mg * la[c] + gv[c] * gl)"),
    ("adjoint_dS_overwritten", "for (size_t q = 0; q < n; ++q) dS[q] += mu[q];",
     "for (size_t q = 0; q < n; ++q) dS[q] = mu[q];"),
    ("adjoint_dr_overwritten", "dr[q] -= gm[0] * gp[0] + gm[1] * gp[1] + gm[2] * gp[2];",
     "dr[q] = -(gm[0] * gp[0] + gm[1] * gp[1] + gm[2] * gp[2]);"),
    ("adjoint_dphi1_closed_form_sign", "return ((z - 1.0) * expm1(z) + z) / (z * z);",
     "return ((z - 1.0) * expm1(z) - z) / (z * z);"),
    ("adjoint_phi1_at_zero", "static double phi1(double z) { return z == 0 ? 1.0 : expm1(z) / z; }",
     "static double phi1(double z) { return z == 0 ? 0.0 : expm1(z) / z; }"),
]

# (name, text in oracle/__init__.py, replacement). Not listed, for lack of a case
# that tells them apart: "Delta m < eps" for "<= eps" (differs only at exact equality),
# and applying the energy rule before the Delta m rule (differs only when both fire
# in the same step).
PY_MUTANTS = [
    ("delta_m_relative_to_new_m", "old2 = (m_old ** 2).sum()", "old2 = (m_new ** 2).sum()"),
    ("delta_m_not_per_unit_time", "/ old2) / dt)", "/ old2))"),
    ("delta_m_of_a_zero_state_undefined", "if old2 == 0:\n        return 0.0", "if old2 < 0:\n        return 0.0"),
    ("run_energy_of_the_new_m", "energies.append(energy(grid, prm, r, m, p))",
     "energies.append(energy(grid, prm, r, m_new, p))"),
    ("run_names_the_wrong_step", "reason, energy_step = 2, k - 1", "reason, energy_step = 2, k"),
    ("run_energy_rule_needs_an_increase", "not energies[-1] < energies[-2]",
     "energies[-1] > energies[-2]"),
    ("run_returns_the_state_before_a_failure", "m, reason = m_new, 3", "reason = 3"),
    ("kbar_array_offdiag_order",
     "return np.array([M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]])",
     "return np.array([M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[1, 2], M[0, 2]])"),
    ("pcg_ignores_the_preconditioner_option",
     "kb = kbar_default(grid, m, r) if precond == 1 else kbar_array(grid.dim, kappa_default(grid, m, r))",
     "kb = kbar_array(grid.dim, kappa_default(grid, m, r))"),
]

CONTROL = ("unchanged_source", None, None)
PY_CONTROL = ("unchanged_python", None, None)


def _build_and_run(base, source, case):
    name, old, new = case
    d = os.path.join(base, name)
    os.makedirs(d)
    shutil.copy(HDR, d)
    text = source if old is None else source.replace(old, new)
    with open(os.path.join(d, "hc_oracle.c"), "w") as f:
        f.write(text)
    lib = os.path.join(d, "libhc_oracle.so")
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                    "-fPIC", "-shared", "-o", lib, "hc_oracle.c", "-lm"], check=True, cwd=d)
    env = dict(os.environ, HC_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider", *PIN_TESTS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode, r.stdout[-3000:] + r.stderr[-1000:]


def _run_python(base, lib, source, case):
    """The pins in a sandbox holding a copy of the tests, the input generators
    and the oracle package with the planted mistake (the C library unchanged)."""
    name, old, new = case
    d = os.path.join(base, name)
    skip = shutil.ignore_patterns("__pycache__", "*.so", "*.tmp")
    shutil.copytree(os.path.join(ROOT, "workloads"), os.path.join(d, "workloads"), ignore=skip)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"), ignore=skip)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(d, "tests", "golden"))
    for f in [os.path.basename(t) for t in PIN_TESTS] + ["conftest.py", "golden_cases.py"]:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(d, "tests", f))
    with open(os.path.join(d, "oracle", "__init__.py"), "w") as f:
        f.write(source if old is None else source.replace(old, new))
    env = dict(os.environ, HC_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider", *PIN_TESTS],
                       cwd=d, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode, r.stdout[-3000:] + r.stderr[-1000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    import oracle
    lib = oracle.build()   # the unchanged library, for the Python mutants
    base = str(tmp_path_factory.mktemp("oracle_mutants"))
    with open(SRC) as f:
        source = f.read()
    with open(PY_SRC) as f:
        py_source = f.read()
    for name, old, _ in MUTANTS:
        assert source.count(old) == 1, f"{name}: the planted text must occur exactly once"
    for name, old, _ in PY_MUTANTS:
        assert py_source.count(old) == 1, f"{name}: the planted text must occur exactly once"
    jobs = [lambda c=c: _build_and_run(base, source, c) for c in [CONTROL] + MUTANTS]
    jobs += [lambda c=c: _run_python(base, lib, py_source, c) for c in [PY_CONTROL] + PY_MUTANTS]
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        done = list(ex.map(lambda job: job(), jobs))
    return {name: (rc, out) for name, rc, out in done}


@pytest.mark.parametrize("name", [CONTROL[0], PY_CONTROL[0]])
def test_harness_control_passes(outcomes, name):
    rc, out = outcomes[name]
    assert rc == 0, out


def test_mutant_names_unique():
    names = [m[0] for m in MUTANTS + PY_MUTANTS] + [CONTROL[0], PY_CONTROL[0]]
    assert len(names) == len(set(names))


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS + PY_MUTANTS])
def test_pins_catch_mutant(outcomes, name):
    rc, out = outcomes[name]
    # 1: some pin failed.  0 would mean the mistake went unnoticed; any other
    # code means the copy crashed or pytest could not run, which proves nothing.
    assert rc == 1, f"{name}: pins exit code {rc}\n{out}"
