"""The oracle's pins have teeth: each plausible mistake, planted in a copy of the
oracle source and compiled on the CPU, makes at least one pin fail.

The copy lives in a temporary directory; the oracle that the other tests use is
never modified.
"""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "cva_oracle.c")

# (name, text in the oracle source, planted replacement, pin that must fail)
PLANTS = [
    ("dropped loss-given-default",
     "V[c * (n + 1) + j] = (1.0 - m->recovery[c]) * exp(-I0[j]) * mp;",
     "V[c * (n + 1) + j] = exp(-I0[j]) * mp;",
     pins.test_cva_identity_independent_constant_hazards),
    ("exposure taken one date early",
     "exp(I0[i]) * V[c * (n + 1) + idx] / N",
     "exp(I0[i]) * V[c * (n + 1) + idx - 1] / N",
     pins.test_cva_identity_independent_constant_hazards),
    ("quanto drift without sigma_r",
     "* m->sigma_chi[e] * m->sigma_r[e];",
     "* m->sigma_chi[e];",
     pins.test_fx_quanto_martingale),
    ("quanto drift dropped",
     "drift -= m->corr[pos_r[e] * F + pos_x[e]]",
     "drift -= 0.0 * m->corr[pos_r[e] * F + pos_x[e]]",
     pins.test_fx_quanto_martingale),
    ("FX drift with the rates swapped",
     "(r[0] - r[e] - 0.5 * sx * sx)",
     "(r[e] - r[0] - 0.5 * sx * sx)",
     pins.test_fx_quanto_martingale),
    ("bond price without its convexity term",
     "+ B * f - s * s / (4.0 * a)",
     "+ B * f - 0.0 * s * s / (4.0 * a)",
     pins.test_discounted_bond_is_a_martingale),
    ("discount integral halved",
     "Iacc += r[0] * ds;",
     "Iacc += 0.5 * r[0] * ds;",
     pins.test_discounted_bond_is_a_martingale),
    ("transposed Cholesky factor",
     "acc += L[a * F + b] * z[b];",
     "acc += L[b * F + a] * z[b];",
     pins.test_factor_increments_have_the_model_correlation),
    ("floating coupon fixed today instead of at the last reset",
     "oracle_zc(m, e, t_minus, t_plus, r_fix)",
     "oracle_zc(m, e, t_minus, t_plus, r_t)",
     pins.test_cva_identity_independent_constant_hazards),
    ("cum-coupon fixing taken today",
     "return 1.0 / oracle_zc(m, e, t_minus, t, r_fix)",
     "return 1.0 / oracle_zc(m, e, t_minus, t, r_t)",
     pins.test_cva_identity_independent_constant_hazards),
    ("default compared with the previous date's integral",
     "if (Lam[c * (n + 1) + j] >= eps)",
     "if (Lam[c * (n + 1) + j - 1] >= eps)",
     pins.test_constant_hazard_survival),
    ("Box-Muller angle halved",
     "z[i0] = rad * cos(2.0 * OR_PI * u2);",
     "z[i0] = rad * cos(OR_PI * u2);",
     pins.test_uniforms_and_normals_are_distributed_correctly),
    ("CIR diffusion without the square root",
     "m->nu[c] * sqrt(gp) * sqds",
     "m->nu[c] * gp * sqds",
     pins.test_cir_survival_closed_form),
]


@pytest.mark.parametrize("name,old,new,pin", PLANTS, ids=[p[0] for p in PLANTS])
def test_planted_mistake_is_caught(name, old, new, pin, tmp_path, oracle_lib):
    src = open(SRC).read()
    assert src.count(old) == 1, f"plant site for {name!r} not found exactly once"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-fno-fast-math", "-ffp-contract=off", str(mutant), "-o", str(so), "-lm"])
    with oracle.use_library(str(so)):
        with pytest.raises(AssertionError):
            if "tmp_path" in pin.__code__.co_varnames[:pin.__code__.co_argcount]:
                pin(oracle_lib, tmp_path)
            else:
                pin(oracle_lib)


# ---- Algorithms 1 and 2 in the Python MLP oracle --------------------------------
from tests import test_oracle_mlp as mlp_pins  # noqa: E402

MLP_SRC = os.path.join(os.path.dirname(oracle.__file__), "mlp.py")

MLP_PLANTS = [
    ("dates iterated in increasing order",
     "for i in sorted(dates, reverse=True):",
     "for i in sorted(dates):",
     mlp_pins.pin_backward_learning_runs_dates_downwards),
    ("every date restarted from the initial parameters",
     "p, best = base_alg(p, Z, y, **kw)",
     "p, best = base_alg(p_init, Z, y, **kw)",
     mlp_pins.pin_backward_learning_warm_starts),
    ("output layer refitted at the last epoch",
     "if epoch == epochs // 2:",
     "if epoch == epochs:",
     mlp_pins.pin_refit_at_half_the_epochs),
    ("output ReLU never switched on",
     "            pos = 1\n",
     "            pos = 0\n",
     mlp_pins.pin_output_relu_after_the_refit),
]


@pytest.mark.parametrize("name,old,new,pin", MLP_PLANTS, ids=[p[0] for p in MLP_PLANTS])
def test_planted_mlp_mistake_is_caught(name, old, new, pin, tmp_path):
    import importlib.util
    src = open(MLP_SRC).read()
    assert src.count(old) == 1, f"plant site for {name!r} not found exactly once"
    path = tmp_path / "mlp_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("mlp_mutant", str(path))
    mutant = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mutant)
    pin(mlp_pins.mlp)   # the unmodified oracle passes
    with pytest.raises(AssertionError):
        pin(mutant)


from tests import test_oracle_dual as dual_pins  # noqa: E402

DUAL_SRC = os.path.join(os.path.dirname(oracle.__file__), "dual.py")

# plausible slips in the forward-mode gradient: each is caught by the value pin or by
# the central-difference pin of tests/test_oracle_dual.py
DUAL_PLANTS = [
    ("product rule with a minus sign",
     "self.d * o.v + o.d * self.v)", "self.d * o.v - o.d * self.v)",
     dual_pins.pin_tangents_are_central_differences),
    ("quotient rule with a plus sign",
     "(self.d * o.v - o.d * self.v) / (o.v * o.v)", "(self.d * o.v + o.d * self.v) / (o.v * o.v)",
     dual_pins.pin_tangents_are_central_differences),
    ("square root derivative without the factor 1/2",
     "x.d / (2.0 * safe)", "x.d / safe",
     dual_pins.pin_tangents_are_central_differences),
    ("positive part passing the tangent where x <= 0",
     "np.where(x.v > 0.0, x.d, 0.0))", "x.d)",
     dual_pins.pin_tangents_are_central_differences),
    ("exponential without the chain factor",
     "return Dual(e, x.d * e)", "return Dual(e, x.d)",
     dual_pins.pin_tangents_are_central_differences),
    ("quanto drift with the wrong sign",
     "drift = drift - sx[e] * sr[e] * q_rho[e]", "drift = drift + sx[e] * sr[e] * q_rho[e]",
     dual_pins.pin_value_is_the_oracle_smooth_cva0),
    ("survival difference taken one date late",
     "share[c] + V * (exp(-Lam_prev[c]) - exp(-Lam[c]))", "share[c] + V * (exp(-Lam[c]) - exp(-Lam[c]))",
     dual_pins.pin_value_is_the_oracle_smooth_cva0),
]


@pytest.mark.parametrize("name,old,new,pin", DUAL_PLANTS, ids=[p[0] for p in DUAL_PLANTS])
def test_planted_dual_mistake_is_caught(name, old, new, pin, tmp_path):
    import importlib.util
    src = open(DUAL_SRC).read()
    assert src.count(old) == 1, f"plant site for {name!r} not found exactly once"
    path = tmp_path / "dual_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("oracle._dual_mutant", str(path))
    mutant = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mutant)
    pin(dual_pins.dual)   # the unmodified oracle passes
    with pytest.raises(AssertionError):
        pin(mutant)
