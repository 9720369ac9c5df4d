"""The pins catch plausible mistakes in the oracle.

Each case copies ``oracle/lsefit_oracle.c``, plants one mistake (a dropped
term, a wrong index, sign or operand, the paper's misprints taken literally),
builds the copy in a temporary directory and runs the pin suite against it in
a separate process.  The suite must fail for every mutant and pass for the
unmodified copy.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lsefit_oracle.c")

MUTANTS = {
    # S_0 read as the "1" printed in the top-left entry of A (Section II)
    "s0_printed_as_one": ("S[0] = (double)n;", "S[0] = 1.0;"),
    # highest T_k dropped
    "drop_T_m": ("if (k <= m) T[k] += p * y[i];", "if (k < m) T[k] += p * y[i];"),
    # highest power sum dropped
    "drop_S_2m": ("if (k > 0) S[k] += p;", "if (k > 0 && k < 2 * m) S[k] += p;"),
    # Hankel index wrong
    "hankel_index": ("for (int k = 0; k < N; ++k) A[j * N + k] = S[j + k];\n        B[j] = T[j];",
                     "for (int k = 0; k < N; ++k) A[j * N + k] = S[j + k + (j == m && k == 1)];\n        B[j] = T[j];"),
    # elimination sign
    "elimination_sign": ("M[i * N + j] -= f * M[k * N + j];", "M[i * N + j] += f * M[k * N + j];"),
    # right-hand side not eliminated
    "rhs_not_eliminated": ("r[i] -= f * r[k];", ";"),
    # transposed operand in back substitution
    "backsub_transposed": ("acc -= M[i * N + j] * z[j];", "acc -= M[j * N + i] * z[j];"),
    # affine map applied as s x - c
    "map_operand": ("double t = map ? map[1] * (x[i] - map[0]) : x[i];\n        double p = 1.0;\n        for (int k = 0; k <= 2 * m; ++k) {",
                    "double t = map ? map[1] * x[i] - map[0] : x[i];\n        double p = 1.0;\n        for (int k = 0; k <= 2 * m; ++k) {"),
    # un-map sign of c
    "unmap_sign": ("acc += Xt[k] * orc_binom(k, j) * pow(s, (double)k) * pow(-c, (double)(k - j));",
                   "acc += Xt[k] * orc_binom(k, j) * pow(s, (double)k) * pow(c, (double)(k - j));"),
    # adjoint: wrong sign of the lambda f' term
    "adjoint_sign": ("dx[i] = sc * (ld * (y[i] - fv) - lv * fd);", "dx[i] = sc * (ld * (y[i] - fv) + lv * fd);"),
    # adjoint: chain-rule factor s dropped
    "adjoint_scale": ("dx[i] = sc * (ld * (y[i] - fv) - lv * fd);", "dx[i] = (ld * (y[i] - fv) - lv * fd);"),
    # adjoint: transpose of the un-map replaced by the un-map itself
    "adjoint_transpose": ("if (map) orc_unmap_transpose(m, map[0], map[1], gX, gt);",
                          "if (map) orc_unmap(m, map[0], map[1], gX, gt);"),
    # Cholesky: diagonal update sign
    "cholesky_sign": ("for (int k = 0; k < j; ++k) d -= Lm[j * N + k] * Lm[j * N + k];",
                      "for (int k = 0; k < j; ++k) d += Lm[j * N + k] * Lm[j * N + k];"),
    # Cholesky: transposed factor in the back substitution
    "cholesky_transposed": ("for (int k = i + 1; k < N; ++k) acc -= Lm[k * N + i] * X[k];",
                            "for (int k = i + 1; k < N; ++k) acc -= Lm[i * N + k] * X[k];"),
    # Chebyshev recurrence with the wrong sign
    "cheb_recurrence_sign": ("2.0 * t * phi[k - 1] - phi[k - 2]", "2.0 * t * phi[k - 1] + phi[k - 2]"),
    # weight applied twice in the normal matrix
    "weight_squared": ("G[j * N + k] += wi * phi[j] * phi[k];", "G[j * N + k] += wi * wi * phi[j] * phi[k];"),
    # weight dropped from the right-hand side
    "weight_dropped_rhs": ("b[j] += wi * phi[j] * y[i];", "b[j] += phi[j] * y[i];"),
    # Chebyshev-to-monomial expansion without the shift by one power
    "cheb_to_mono_shift": ("(j > 0 ? 2.0 * P[(k - 1) * N + j - 1] : 0.0)", "(j > 0 ? 2.0 * P[(k - 1) * N + j] : 0.0)"),
    # residual diagnostics: V^T y accumulated instead of V^T r
    "residual_vtr_operand": ("vtr[k] += phi[k] * r;", "vtr[k] += phi[k] * y[i];"),
    # residual sign reversed (the SSE alone cannot see it)
    "residual_sign": ("const double r = y[i] - f;", "const double r = f - y[i];"),
    # residual evaluation drops the constant term
    "eval_drop_a0": ("acc += X[j] * p;\n            p *= x[i];\n        }\n        f[i] = acc;",
                     "if (j) acc += X[j] * p;\n            p *= x[i];\n        }\n        f[i] = acc;"),
}


def _run_pins(src_path, build_dir):
    env = dict(os.environ)
    env["LSEFIT_ORACLE_SOURCE"] = src_path
    env["LSEFIT_ORACLE_BUILD_DIR"] = build_dir
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
           os.path.join(ROOT, "tests", "test_oracle_pins.py")]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def _mutant_source(tmp_path, name, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(text.replace(old, new))
    return str(path)


def test_unmutated_copy_passes(tmp_path):
    path = tmp_path / "copy.c"
    path.write_text(open(SRC).read())
    r = _run_pins(str(path), str(tmp_path / "build"))
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    path = _mutant_source(tmp_path, name, old, new)
    r = _run_pins(path, str(tmp_path / "build"))
    assert r.returncode != 0, f"mutant {name} survived the pins"
    assert "FAILED" in r.stdout or "Error" in r.stdout, r.stdout[-2000:]
