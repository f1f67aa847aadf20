"""Plant mistakes in a copy of the oracle (on the CPU) and check that the pins
catch every one: a pin set that a dropped term, a wrong sign or a transposed
operand slips through would not pin anything."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "dpsr_oracle.c")

# (name, exact text in the oracle, replacement)
MUTANTS = [
    ("dft_sign", "double ang = sign * 2.0 * kPi", "double ang = -sign * 2.0 * kPi"),
    ("no_gaussian", "double g = exp(-2.0 * sigma * sigma * f2", "double g = 1.0 + 0.0 * exp(-2.0 * sigma * sigma * f2"),
    ("gaussian_no_r2", "f2 / ((double)r * (double)r))", "f2 / ((double)r))"),
    ("laplacian_factor", "(-2.0 * kPi * u2)", "(-kPi * u2)"),
    ("transposed_u", "(I * (freq(k[a], r) / box[a]))", "(I * (freq(k[(a + 1) % 3], r) / box[a]))"),
    ("nyquist_norm", "k[d] == r / 2 ? (double)(r / 2)", "k[d] == r / 2 ? 0.0"),
    ("unshifted_scale", "S->s = S->chip[0] - S->mu;", "S->s = S->chip[0];"),
    ("weights_swapped", "f[d] = del[d] ? t[d] : 1.0 - t[d];", "f[d] = del[d] ? 1.0 - t[d] : t[d];"),
    ("bwd_drop_W", "Ghat[j] = alpha * dchi[j] + (mu_bar / (double)N) * W[j];", "Ghat[j] = alpha * dchi[j];"),
    ("bwd_dw_sign", "df[d] = del[d] ? (double)r : -(double)r;", "df[d] = del[d] ? -(double)r : (double)r;"),
    ("bwd_no_conj", "tmp[j] = conj(spectral_H(a, k, r, sigma, box)) * Ghat[j];", "tmp[j] = spectral_H(a, k, r, sigma, box) * Ghat[j];"),
    ("bwd_s_bar_sign", "const double s_bar = -kM * sgn", "const double s_bar = kM * sgn"),
    ("box_u_not_scaled", "u2 += (f / box[d]) * (f / box[d]);", "u2 += f * f;"),
    ("box_grad_not_scaled", "dpts[3 * i + d] /= box[d];", "dpts[3 * i + d] /= 1.0;"),
    ("box_gaussian_in_u", "sigma * sigma * f2 /", "sigma * sigma * u2 /"),
    ("box_coords_axis0", "u[3 * i + d] = pts[3 * i + d] / box[d];", "u[3 * i + d] = pts[3 * i + d] / box[0];"),
    ("bwd_mean_term_is_rest", "if (dpts_mean) dpts_mean[3 * i + d] = gm[d];",
     "if (dpts_mean) dpts_mean[3 * i + d] = gc[d];"),
    ("bwd_mean_term_no_mu_bar", "gm[d] += (mu_bar / (double)N) * st.dw[v][d]",
     "gm[d] += (1.0 / (double)N) * st.dw[v][d]"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", str(lib), str(mut), "-lm"],
                   check=True)
    env = dict(os.environ, ORACLE_LIB=str(lib), OMP_NUM_THREADS="2")
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(HERE, "test_oracle_pins.py")],
                         env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"planted mistake {name} passed every pin:\n{res.stdout[-2000:]}"
