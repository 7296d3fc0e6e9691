"""The oracle's pins must reject a wrong oracle.

Each mutant below plants one plausible mistake in a copy of the oracle: a
dropped term, a wrong sign, a wrong index, a transposed or swapped operand, a
wrong weight or coefficient. For oracle/oracle.c the copy is compiled beside
the test and the pin suites of the C oracle (tests/test_oracle_{model,
smoother,iterated,lm}.py) run against it in a child process (oracle/
__init__.py loads the library that PES_ORACLE_LIBRARY names); for
oracle/learned_init.py the child process imports the mutated copy in its
place and runs tests/test_oracle_learned_init.py. At least one pin has to
fail. Unmodified copies, run the same way, have to pass them all, which also
shows that the child processes use the copies.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")
PIN_SUITES = [os.path.join(ROOT, "tests", f"test_oracle_{n}.py") for n in ("model", "smoother", "iterated", "lm")]
LI_PINS = os.path.join(ROOT, "tests", "test_oracle_learned_init.py")

# (name, anchor, old, new): `old` is replaced by `new` at its first occurrence
# after the first occurrence of `anchor` (the function it sits in).
MUTANTS = [
    # model (Sec. 5: coordinated turn, bearings, noise)
    ("ct_f_sign", "void orc_ct_f(", "out[0] = x[0] + A1 * x[2] - A2 * x[3];", "out[0] = x[0] + A1 * x[2] + A2 * x[3];"),
    ("ct_f_rotation", "void orc_ct_f(", "out[3] = s * x[2] + c * x[3];", "out[3] = -s * x[2] + c * x[3];"),
    ("ct_series_coefficient", "static void ct_coeffs(", "*A2 = dt * a * (0.5 - a2 / 24.0", "*A2 = dt * a * (0.5 - a2 / 12.0"),
    ("ct_closed_form_derivative", "static void ct_coeffs(", "*dA1 = (a * c - s) / (w * w);",
     "*dA1 = (a * c + s) / (w * w);"),
    ("ct_jacobian_entry", "void orc_ct_jacobian(", "F[2 * 5 + 4] = -dt * s * x[2] - dt * c * x[3];",
     "F[2 * 5 + 4] = -dt * s * x[2] + dt * c * x[3];"),
    ("bearing_arguments_swapped", "void orc_bearings_h(", "atan2(x[1] - s[2 * r + 1], x[0] - s[2 * r])",
     "atan2(x[0] - s[2 * r], x[1] - s[2 * r + 1])"),
    ("bearing_jacobian_sign", "void orc_bearings_jacobian(", "H[r * 5 + 0] = -dy / rho2;", "H[r * 5 + 0] = dy / rho2;"),
    ("process_noise_coefficient", "void orc_process_noise(", "m->q_c * dt * dt * dt / 3.0;",
     "m->q_c * dt * dt * dt / 2.0;"),
    ("process_noise_turn_rate", "void orc_process_noise(", "Q[4 * 5 + 4] = m->q_w * dt;", "Q[4 * 5 + 4] = m->q_c * dt;"),
    ("measurement_noise_not_squared", "void orc_measurement_noise(", "R[0] = m->r_std * m->r_std;",
     "R[0] = m->r_std;"),
    ("wrap_range", "double orc_wrap(", "floor((a + ORC_PI) / (2.0 * ORC_PI))", "floor(a / (2.0 * ORC_PI))"),
    # linear algebra
    ("mmt_transposed_operand", "static void mmt(", "B[j * m + l]", "B[l * m + j]"),
    ("chol_solve_back_substitution", "static void chol_solve(", "s -= L[l * n + i] * X[l * r + c];",
     "s -= L[i * n + l] * X[l * r + c];"),
    # cubature SLR (Eqs. 7-9)
    ("cubature_weight", "int orc_slr(", "const double w = 1.0 / (2.0 * NX);", "const double w = 1.0 / NX;"),
    ("cubature_spread", "int orc_slr(", "const double scale = sqrt((double)NX);", "const double scale = (double)NX;"),
    ("slr_lambda_dropped_term", "int orc_slr(", "Lam[r] = Phi[r] - GPG[r];", "Lam[r] = Phi[r];"),
    ("slr_offset_dropped_term", "int orc_slr(", "offset[r] = zbar[r] - Gx[r];", "offset[r] = zbar[r];"),
    ("slr_slope_transposed", "int orc_slr(", "G[r * NX + i] = Gt[i * nz + r];", "G[r * NX + i] = Gt[r * nz + i];"),
    ("slr_no_unwrap", "int orc_slr(", "Z[j][r] = ref[r] + orc_wrap(Z[j][r] - ref[r]);", "Z[j][r] = Z[j][r];"),
    ("slr_covariance_centre", "int orc_slr(", "Psi[i * nz + r] += w * (X[j][i] - xbar[i]) * (Z[j][r] - zbar[r]);",
     "Psi[i * nz + r] += w * X[j][i] * (Z[j][r] - zbar[r]);"),
    # unscented and Gauss-Hermite rules
    ("unscented_beta_dropped", "int orc_slr_unscented(", "Wc[0] = Wm[0] + 1.0 - a * a + m->ut_beta;",
     "Wc[0] = Wm[0] + 1.0 - a * a;"),
    ("unscented_lambda", "int orc_slr_unscented(", "const double lambda = a * a * (n + m->ut_kappa) - n;",
     "const double lambda = a * (n + m->ut_kappa) - n;"),
    ("unscented_weight", "int orc_slr_unscented(", "Wm[j] = Wc[j] = 1.0 / (2.0 * (n + lambda));",
     "Wm[j] = Wc[j] = 1.0 / (n + lambda);"),
    ("gauss_hermite_weights", "int orc_slr_gauss_hermite(", "{1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0}",
     "{1.0 / 4.0, 1.0 / 2.0, 1.0 / 4.0}"),
    ("gauss_hermite_nodes", "int orc_slr_gauss_hermite(", "{-sqrt(3.0), 0.0, sqrt(3.0)}",
     "{-sqrt(2.0), 0.0, sqrt(2.0)}"),
    # linearisation of a step (Eq. 10, Q' and R')
    ("taylor_offset_dropped_term", "int orc_linearize(", "c[5 * k + i] = fx[i] - Fx[i];", "c[5 * k + i] = fx[i];"),
    ("taylor_observation_offset_sign", "int orc_linearize(", "d[2 * k + r] = hx[r] - Hx[r];",
     "d[2 * k + r] = hx[r] + Hx[r];"),
    ("q_prime_drops_lambda", "int orc_linearize(", "Qp[25 * k + i] = Q[i] + Lam[i];", "Qp[25 * k + i] = Q[i];"),
    ("r_prime_drops_omega", "int orc_linearize(", "Rp[4 * k + i] = R[i] + Om[i];", "Rp[4 * k + i] = R[i];"),
    ("measurement_not_unwrapped", "int orc_linearize(", "angles(m) ? hx[r] + orc_wrap(y[2 * k + r] - hx[r]) : y[2 * k + r]",
     "y[2 * k + r]"),
    # Kalman filter and RTS smoother (the definition)
    ("kf_transition_index", "int orc_kf_rts_damped(", "const double* Fk = F + 25 * (k - 1);", "const double* Fk = F + 25 * k;"),
    ("kf_process_noise_index", "int orc_kf_rts_damped(", "P_[i] += Qp[25 * (k - 1) + i];", "P_[i] += Qp[25 * k + i];"),
    ("kf_innovation_sign", "int orc_kf_rts_damped(", "v[r] = y[2 * k + r] - Hm[r] - d[2 * k + r];",
     "v[r] = y[2 * k + r] - Hm[r] + d[2 * k + r];"),
    ("kf_covariance_update_sign", "int orc_kf_rts_damped(", "Pf[25 * k + i] = P_[i] - KSK[i];",
     "Pf[25 * k + i] = P_[i] + KSK[i];"),
    ("rts_gain_not_transposed", "int orc_kf_rts_damped(", "G[i * 5 + j] = Gt[j * 5 + i];", "G[i * 5 + j] = Gt[i * 5 + j];"),
    ("rts_mean_sign", "int orc_kf_rts_damped(", "xs[5 * k + i] = xf[5 * k + i] + Gdm[i];",
     "xs[5 * k + i] = xf[5 * k + i] - Gdm[i];"),
    ("rts_covariance_sign", "int orc_kf_rts_damped(", "Ps[25 * k + i] = Pf[25 * k + i] + GdPG[i];",
     "Ps[25 * k + i] = Pf[25 * k + i] - GdPG[i];"),
    ("damping_variance", "static int damp_update(", "S[i * NX + i] += 1.0 / lambda;", "S[i * NX + i] += lambda;"),
    ("loglik_drops_log_det", "int orc_kf_loglik(", "ll += -0.5 * (q + log(det))", "ll += -0.5 * q"),
    # the iteration (Sec. 3)
    ("iteration_keeps_prior_covariance", "int orc_iterated_smoother(", "memcpy(P_out, Ps, sizeof(double) * 25 * N);",
     ";"),
    ("update_norm_of_old_iterate", "int orc_iterated_smoother(", "den += xs[5 * k + i] * xs[5 * k + i];",
     "den += x_out[5 * k + i] * x_out[5 * k + i] * 1e-4;"),
    # MAP objective and Levenberg-Marquardt
    ("map_cost_drops_prior", "int orc_map_cost(", "for (int i = 0; i < NX; ++i) J += 0.5 * e[i] * t[i];",
     "for (int i = 0; i < NX; ++i) J += 0.0 * e[i] * t[i];"),
    ("map_cost_residual_not_wrapped", "int orc_map_cost(", "if (angles(m)) r[i] = orc_wrap(r[i]);", ";"),
    ("lm_accept_raises_damping", "int orc_iterated_smoother_lm(", "lam[b] /= nu;", "lam[b] *= nu;"),
    ("lm_accepts_any_step", "int orc_iterated_smoother_lm(", "if (Jnew[b] < Jcur[b]) {", "if (1) {"),
    # the paper's elements and operators (Eqs. 13-19)
    ("filter_element_gain_sign", "int orc_filter_element(", "e->b[i] = c[i] + Kv[i];", "e->b[i] = c[i] - Kv[i];"),
    ("filter_element_eta_drops_s_inverse", "int orc_filter_element(", "mtv(NX, NY, HF, Siv, e->eta);",
     "mtv(NX, NY, HF, v, e->eta);"),
    ("combine_drops_c_eta", "int orc_filter_combine(", "for (int i = 0; i < NX; ++i) t1[i] += ei->b[i];",
     "for (int i = 0; i < NX; ++i) t1[i] = ei->b[i];"),
    ("combine_drops_j_i", "int orc_filter_combine(", "r.J[i] = AitMtJA[i] + ei->J[i];", "r.J[i] = AitMtJA[i];"),
    ("combine_cj_order", "int orc_filter_combine(", "mm(NX, NX, NX, ei->C, ej->J, CJ);", "mm(NX, NX, NX, ej->J, ei->C, CJ);"),
    ("smoother_element_sign", "int orc_smoother_element(", "e->g[i] = xf[i] - Em[i];", "e->g[i] = xf[i] + Em[i];"),
    ("smoother_combine_swapped", "void orc_smoother_combine(", "mv(NX, NX, ei->E, ej->g, Eg);",
     "mv(NX, NX, ej->E, ei->g, Eg);"),
    ("smoother_combine_wrong_l", "void orc_smoother_combine(", "r.L[i] = ELE[i] + ei->L[i];", "r.L[i] = ELE[i] + ej->L[i];"),
    ("filter_element_a_drops_gain", "int orc_filter_element(", "mm(NX, NX, NX, IKH, F, e->A);",
     "memcpy(e->A, F, sizeof(double) * 25);"),
    ("filter_element_c_drops_gain", "int orc_filter_element(", "mm(NX, NX, NX, IKH, Qp, e->C);",
     "memcpy(e->C, Qp, sizeof(double) * 25);"),
    ("prior_element_drops_covariance", "void orc_filter_prior_element(", "memcpy(e->C, P0, sizeof(double) * 25);",
     "memset(e->C, 0, sizeof(double) * 25);"),
    ("combine_eta_sign", "int orc_filter_combine(", "t1[i] = ej->eta[i] - t1[i];", "t1[i] = ej->eta[i] + t1[i];"),
    ("combine_drops_c_j", "int orc_filter_combine(", "r.C[i] = AjMCAt[i] + ej->C[i];", "r.C[i] = AjMCAt[i];"),
    ("smoother_element_l_sign", "int orc_smoother_element(", "e->L[i] = Pf[i] - EFP[i];", "e->L[i] = Pf[i] + EFP[i];"),
    ("smoother_combine_e_order", "void orc_smoother_combine(", "mm(NX, NX, NX, ei->E, ej->E, r.E);",
     "mm(NX, NX, NX, ej->E, ei->E, r.E);"),
    ("taylor_transition_about_next_state", "int orc_linearize(", "model_f_jac(m, xk, F + 25 * k);",
     "model_f_jac(m, xk + 5, F + 25 * k);"),
    ("kf_gain_drops_s_inverse", "int orc_kf_rts_damped(", "mm(NX, NY, NY, PHt, Sinv, K);", "mm(NX, NY, NY, PHt, S, K);"),
    ("iteration_about_filtered_means", "int orc_iterated_smoother(", "memcpy(x_out, xs, sizeof(double) * 5 * N);",
     "memcpy(x_out, xf, sizeof(double) * 5 * N);"),
    ("loglik_normalising_constant", "int orc_kf_loglik(", "- 0.5 * NY * log_2pi;", "- 0.5 * log_2pi;"),
]

# the same for oracle/learned_init.py
LI_MUTANTS = [
    ("bf16_ties_away", "def bf16(", "(u + 0x7FFF + ((u >> 16) & 1))", "(u + 0x8000)"),
    ("features_sin_for_cos", "def features(", "phi[1:, 1] = np.cos(yy[0, 1:])", "phi[1:, 1] = np.sin(yy[0, 1:])"),
    ("features_head_marker", "def features(", "phi[0, 5] = 1.0", "phi[0, 4] = 1.0"),
    ("shift_direction", "def shift(", "s[:n - d] = h[d:]", "s[d:] = h[:n - d]"),
    ("conv_flipped_taps", "def conv(", "shift(h, j - TAPS // 2)", "shift(h, TAPS // 2 - j)"),
    ("conv_weight_transposed", "def conv(", "@ W[:, :, j].T", "@ W[:, :, j]"),
    ("head_without_relu", "def forward(", "z = _r(np.maximum(h[-1] @ W5.T + b5, 0.0), rounding)",
     "z = _r(h[-1] @ W5.T + b5, rounding)"),
    ("nominal_drops_scale", "def initial_nominal(", "np.asarray(sigma)[None, :] * o", "o"),
    ("loss_gradient_scale", "def loss_and_grad(", "_r(2.0 * e / (NOUT * n_total), rounding)",
     "_r(2.0 * e / n_total, rounding)"),
    ("head_gradient_drops_mask", "def loss_and_grad(", "dz = _r((dO @ W6) * (z > 0), rounding)",
     "dz = _r(dO @ W6, rounding)"),
    ("output_bias_gradient", "def loss_and_grad(", "grads[NCONV + 1][1][...] += dO.sum(axis=0)",
     "grads[NCONV + 1][1][...] += dO.sum(axis=1).sum()"),
    ("conv_bias_gradient_dropped", "def loss_and_grad(", "gb += dh.sum(axis=0)", "gb += 0.0"),
    ("conv_weight_gradient_taps", "def loss_and_grad(", "gW[:, :, j] += dh.T @ shift(h[l], j - TAPS // 2)",
     "gW[:, :, j] += dh.T @ shift(h[l], TAPS // 2 - j)"),
    ("backward_conv_direction", "def loss_and_grad(", "back += shift(dh, TAPS // 2 - j) @ W[:, :, j]",
     "back += shift(dh, j - TAPS // 2) @ W[:, :, j]"),
    ("backward_relu_mask_of_next_layer", "def loss_and_grad(", "dh = _r(back * (h[l] > 0), rounding)",
     "dh = _r(back * (h[l + 1] > 0), rounding)"),
    ("adam_no_bias_correction", "def step(", "mhat = self.m / (1 - self.b1 ** self.t)", "mhat = self.m"),
    ("adam_second_moment_not_squared", "def step(", "(1 - self.b2) * g * g", "(1 - self.b2) * np.abs(g)"),
    ("adam_eps_inside_root", "def step(", "(np.sqrt(vhat) + self.eps)", "np.sqrt(vhat + self.eps)"),
]

# Runs the learned-initialiser pins with the module at argv[1] standing in for
# oracle.learned_init.
LI_RUNNER = """
import importlib.util, sys
spec = importlib.util.spec_from_file_location("oracle.learned_init", sys.argv[1])
mod = importlib.util.module_from_spec(spec)
sys.modules["oracle.learned_init"] = mod
spec.loader.exec_module(mod)
import oracle
oracle.learned_init = mod
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", sys.argv[2]]))
"""


def mutate(src: str, anchor: str, old: str, new: str) -> str:
    a = src.index(anchor)
    i = src.index(old, a)
    return src[:i] + new + src[i + len(old):]


def build(src: str, where: str) -> str:
    os.makedirs(where, exist_ok=True)
    shutil.copy(os.path.join(ORACLE_DIR, "oracle.h"), where)
    with open(os.path.join(where, "oracle.c"), "w") as f:
        f.write(src)
    lib = os.path.join(where, "liboracle.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", lib, os.path.join(where, "oracle.c"),
                           "-lm"])
    return lib


def _tail(r) -> str:
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    return lines[-1] if lines else r.stderr[-200:]


def run_pins(lib: str) -> tuple[int, str]:
    env = dict(os.environ, PES_ORACLE_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        *PIN_SUITES], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, _tail(r)


def run_li_pins(module: str) -> tuple[int, str]:
    r = subprocess.run([sys.executable, "-c", LI_RUNNER, module, LI_PINS], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    return r.returncode, _tail(r)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    src = open(os.path.join(ORACLE_DIR, "oracle.c")).read()
    li_src = open(os.path.join(ORACLE_DIR, "learned_init.py")).read()
    base = tmp_path_factory.mktemp("mutants")

    def one(item):
        kind, (name, anchor, old, new) = item
        where = str(base / kind / name)
        if kind == "c":
            text = src if name == "control" else mutate(src, anchor, old, new)
            return (kind, name), run_pins(build(text, where))
        text = li_src if name == "control" else mutate(li_src, anchor, old, new)
        os.makedirs(where, exist_ok=True)
        path = os.path.join(where, "learned_init.py")
        with open(path, "w") as f:
            f.write(text)
        return (kind, name), run_li_pins(path)

    control = ("control", "", "", "")
    items = [("c", control)] + [("c", m) for m in MUTANTS] + [("li", control)] + [("li", m) for m in LI_MUTANTS]
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        return dict(ex.map(one, items))


@pytest.mark.parametrize("path,mutants", [("oracle.c", MUTANTS), ("learned_init.py", LI_MUTANTS)])
def test_mutations_apply_to_distinct_sites(path, mutants):
    src = open(os.path.join(ORACLE_DIR, path)).read()
    names = [m[0] for m in mutants]
    assert len(set(names)) == len(names)
    for name, anchor, old, new in mutants:
        assert src.count(anchor) == 1, name
        assert old in src[src.index(anchor):], name
        assert mutate(src, anchor, old, new) != src, name


@pytest.mark.parametrize("kind", ["c", "li"])
def test_unmodified_copy_passes_the_pins(outcomes, kind):
    rc, tail = outcomes[(kind, "control")]
    assert rc == 0, tail


@pytest.mark.parametrize("kind,name", [("c", m[0]) for m in MUTANTS] + [("li", m[0]) for m in LI_MUTANTS])
def test_pins_reject_the_mutant(outcomes, kind, name):
    rc, tail = outcomes[(kind, name)]
    assert rc == 1, f"{name} survived the pins ({tail})"
