"""Plant mistakes in copies of the oracle and check that the pins catch each.

Every mutant is a one-line textual change of ``oracle/hawkes_oracle.c`` of the
kind a plausible implementation error makes (a dropped indicator or term, a
wrong sign, exponent or index, a transposed operand).  Each is compiled into a
temporary directory and must fail at least one pin; the real oracle is never
modified."""
import os
import subprocess

import pytest

import oracle
import oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "hawkes_oracle.c")

MUTANTS = {
    "background_indicator_dropped": ("    if (tn == tm)\n        return 0.0;\n", ""),
    "selfexcitation_indicator_reversed": ("if (!(tm < tn))", "if (!(tm > tn))"),
    "tau_x_power_off_by_one": ("pow(p->tau_x, (double)d) * p->tau_t", "pow(p->tau_x, (double)(d - 1)) * p->tau_t"),
    "h_power_dropped": ("p->theta * p->omega / pow(p->h, (double)d)", "p->theta * p->omega"),
    "time_kernel_bandwidth_squared_dropped": ("phi_d(dt * dt / (p->tau_t * p->tau_t), 1)", "phi_d(dt * dt / p->tau_t, 1)"),
    "gradient_sign": ("nadd(&acc[k], coef * (xm[k] - xn[k]));", "nadd(&acc[k], coef * (xn[k] - xm[k]));"),
    "gradient_rates_transposed": ("(xi_nm / lam[row] + xi_mn / lam[m]) / h2", "(xi_nm / lam[m] + xi_mn / lam[row]) / h2"),
    "gradient_bandwidth_swapped": ("(xi_nm / lam[row] + xi_mn / lam[m]) / h2", "(xi_nm / lam[row] + xi_mn / lam[m]) / tx2"),
    "Lambda_selfexcitation_sign": ("p->theta * (exp(-p->omega * a) - 1.0);", "p->theta * (1.0 - exp(-p->omega * a));"),
    "Lambda_decay_dropped": ("p->theta * (exp(-p->omega * a) - 1.0);", "p->theta * (exp(-a) - 1.0);"),
    "Lambda_lower_limit_dropped": ("(Phi(a / p->tau_t) - Phi(-t[i] / p->tau_t))", "(Phi(a / p->tau_t) - 0.5)"),
    "window_end_is_last_not_max": ("        if (t[i] > T)\n            T = t[i];\n", ""),
    "theta_grad_Phi_term_dropped": ("double l0 = -(Phi(a_ / tt) - Phi(-t[i] / tt));", "double l0 = 0.0;"),
    "theta_scale_Lambda_part_dropped": ("            nadd(&sm[3], fabs(l3));\n", ""),
    "theta_scale_piece_sign": ("nadd(&b[1], mu * (r2 / (tx * tx * tx) + (double)d / tx));",
                               "nadd(&b[1], mu * (r2 / (tx * tx * tx) - (double)d / tx));"),
    "omega_grad_sign": ("nadd(&a[4], xi * (1.0 / w - dt));", "nadd(&a[4], xi * (1.0 / w + dt));"),
    "tau_t_grad_boundary_term_dropped": ("phi_d(t[i] * t[i] / (tt * tt), 1) * t[i]) /", "0.0) /"),
    "rate_parts_swapped": ("nadd(&s_mu, mu);\n        nadd(&s_xi, xi);", "nadd(&s_mu, xi);\n        nadd(&s_xi, mu);"),
    "bmds_normalizer_sign": ("*out_loglik = c * log(sigma2) - nval(&tot);", "*out_loglik = -c * log(sigma2) - nval(&tot);"),
    "bmds_log_Phi_dropped": ("(2.0 * sigma2) + log(Phi_z));", "(2.0 * sigma2));"),
    "bmds_gradient_ratio_unscaled": ("ratio / sigma;", "ratio;"),
    "bmds_sigma_derivative_halved": ("ratio * delta / (2.0 * sigma2 * sigma));", "ratio * delta / (4.0 * sigma2 * sigma));"),
    "bmds_coincident_guard_dropped": ("if (grad && delta > 0.0) {", "if (grad) {"),
    "lens_segment_sign": ("x_minus_sin(2.0 * th1) + 0.5 * rho * rho", "x_minus_sin(2.0 * th1) - 0.5 * rho * rho"),
    "circle_success_factor_dropped": ("nadd(&lq, (log_success(A_y, rho, tries) - log(A_y)) - (log_success(A_x, rho, tries) - log(A_x)));",
                                      "nadd(&lq, log(A_x) - log(A_y));"),
    "circle_radius_not_sqrt": ("const double r = rho * sqrt(u[(b * tries + k) * 2]);",
                               "const double r = rho * u[(b * tries + k) * 2];"),
    "box_ratio_inverted": ("nadd(&lq, log(Zx) - log(Zy));", "nadd(&lq, log(Zy) - log(Zx));"),
    "bmds_hmc_gradient_sign": ("        g[i] += gb[i];", "        g[i] -= gb[i];"),
    "bmds_hmc_potential_dropped": ("    *ell += lb;", "    *ell += 0.0 * lb;"),
    "hmc_full_step_kicks": ("double half = 0.5 * eps;", "double half = eps;"),
    "hmc_reflection_keeps_momentum": ("            *x = 2.0 * lo - *x;\n            *pm = -*pm;", "            *x = 2.0 * lo - *x;"),
    "hmc_accept_inequality_reversed": ("log_u < H0 - H1) ? 1 : 0", "log_u > H0 - H1) ? 1 : 0"),
    "hmc_kinetic_energy_unhalved": ("nadd(&k1, 0.5 * (pm[i] * pm[i]));", "nadd(&k1, (pm[i] * pm[i]));"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} is not unique in the source"
    mutated = src.replace(old, new, 1)
    cpath = tmp_path / f"{name}.c"
    cpath.write_text(mutated)
    so = tmp_path / f"lib{name}.so"
    cmd = oracle.compile_command(str(so))
    cmd[cmd.index(oracle._SRC)] = str(cpath)
    subprocess.run(cmd, check=True)
    return oracle.Oracle(oracle.load_library(str(so)))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    o = _build_mutant(tmp_path, name, old, new)
    caught = []
    for pin_name, pin in pins.ALL_PINS.items():
        if pin_name == "space_time_quadrature":
            continue  # slow; the other pins suffice for every mutant
        try:
            ok, _ = pin(o)
        except Exception:
            ok = False
        if not ok:
            caught.append(pin_name)
    assert caught, f"mutant {name} passed every pin"
