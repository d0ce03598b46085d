"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of oracle.c (on the CPU, in a temp
directory), builds it, and runs the oracle pin modules against it in a
subprocess; the run must fail.  The unmodified oracle passes the same pins
(the other test modules), so a failure here means the pins are too weak.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
PINS = ["tests/test_oracle_gll.py", "tests/test_oracle_geometry.py", "tests/test_oracle_axlocal.py",
        "tests/test_oracle_gs.py", "tests/test_oracle_pcg.py"]

MUTATIONS = {
    "transposed_dhat_in_second_pass": ("y0 += D[n * N1 + i] * r", "y0 += D[i * N1 + n] * r"),
    "dropped_t_contraction": ("y[i + j * N1 + k * N1 * N1] = y0 + y1 + y2;", "y[i + j * N1 + k * N1 * N1] = y0 + y1;"),
    "sign_of_g02_in_r": ("r[l] = g00 * x0 + g01 * x1 + g02 * x2;", "r[l] = g00 * x0 + g01 * x1 - g02 * x2;"),
    "wrong_factor_in_s": ("s[l] = g01 * x0 + g11 * x1 + g12 * x2;", "s[l] = g02 * x0 + g11 * x1 + g12 * x2;"),
    "wrong_fiber_index_x1": ("x1 += D[j * N1 + n] * x[i + n * N1 + k * N1 * N1];", "x1 += D[j * N1 + n] * x[n + i * N1 + k * N1 * N1];"),
    "jacobian_scale": ("J[3 * c + d] = acc / 8.0;", "J[3 * c + d] = acc / 4.0;"),
    "inverse_product_order": ("acc += inv[3 * p + m] * inv[3 * q + m];", "acc += inv[3 * m + p] * inv[3 * m + q];"),
    "weight_dropped": ("const double s = W * det;", "const double s = det;"),
    "gll_weight_formula": ("w[i] = (double)(2.0L / ((long double)N * (N + 1) * LN[i] * LN[i]));",
                           "w[i] = (double)(2.0L / ((long double)N * (N + 2) * LN[i] * LN[i]));"),
    "dhat_corner": ("else if (i == 0) d = -(long double)N * (N + 1) / 4.0L;", "else if (i == 0) d = -(long double)N * (N + 1) / 2.0L;"),
    "map_vertex_order": ("kron3(tv, sv, rv, row);", "kron3(rv, sv, tv, row);"),
    "gather_overwrites": ("yg[gid[m]] += Yl[m];", "yg[gid[m]] = Yl[m];"),
    "cg_beta_inverted": ("const double beta = rz_new / rz;", "const double beta = rz / rz_new;"),
    "cg_mask_dropped": ("      if (mask[g]) w[g] = 0.0;", "      if (mask[g]) w[g] = w[g];"),
    "diag_wrong_entry": ("diag[(int64_t)n3 * e + l] = y[l];", "diag[(int64_t)n3 * e + l] = y[(l + 1) % n3];"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", str(lib), str(mut), "-lm"])
    env = dict(os.environ, ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + PINS,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "pins did not catch mutation %s:\n%s" % (name, r.stdout[-2000:])
