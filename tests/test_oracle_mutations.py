"""The oracle's pins must be strong enough to catch a plausible mistake.

Each case copies harp_oracle.c, plants one mistake (a dropped sign, a wrong
index, a transposed operand), compiles the copy on the CPU and runs the pin
suite against it: the suite has to fail. The real oracle is never edited.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "harp_oracle.c")
PINS = ["tests/test_oracle_fill.py", "tests/test_oracle_solve.py", "tests/test_oracle_grad.py",
        "tests/test_oracle_eep.py"]

MUTATIONS = {
    "phase_sign": ("const cplx phase = cexp(-I * k * r); /* e^{-jkr}",
                   "const cplx phase = cexp(I * k * r); /* e^{-jkr}"),
    "harmonic_sign": ("for (int p = -P; p <= P; ++p) eh[p + P] = cexp(I * (double)p * alpha);",
                      "for (int p = -P; p <= P; ++p) eh[p + P] = cexp(-I * (double)p * alpha);"),
    "power_off_by_one": ("for (int q = 0; q <= Q; ++q) dq[q] = pow(d, (double)q);",
                         "for (int q = 0; q <= Q; ++q) dq[q] = pow(d, (double)(q + 1));"),
    "coef_T_S_transposed": ("const cplx* c = coef + ((size_t)T * Nm + S) * np * nq;\n      cplx B",
                            "const cplx* c = coef + ((size_t)S * Nm + T) * np * nq;\n      cplx B"),
    "alpha_reversed": ("      const double dx = pos[2 * m] - pos[2 * n];\n      const double dy = pos[2 * m + 1] - pos[2 * n + 1];\n      if (dx == 0.0",
                       "      const double dx = pos[2 * n] - pos[2 * m];\n      const double dy = pos[2 * n + 1] - pos[2 * m + 1];\n      if (dx == 0.0"),
    "far_field_power": ("gpat * phase / r;", "gpat * phase / (r * r);"),
    "lu_update_sign": ("for (int i = k + 1; i < N; ++i) aj[i] -= l[i] * u;",
                       "for (int i = k + 1; i < N; ++i) aj[i] += l[i] * u;"),
    "pivot_not_largest": ("      if (v > best) {", "      if (best == 0.0 && v > best) {"),
    "transpose_swap_order": ("/* x = P^T z: undo the swaps in reverse order. */\n      for (int k = N - 1; k >= 0; --k) {",
                             "/* x = P^T z: undo the swaps in reverse order. */\n      for (int k = 0; k < N; ++k) {"),
    "grad_alpha_sign": ("const cplx zx = a * (dx / r) + b * (-dy / (r * r));",
                        "const cplx zx = a * (dx / r) + b * (dy / (r * r));"),
    "grad_dr_power": ("(double)q * pow(d, (double)(q - 1)) * dd_dr", "(double)q * pow(d, (double)q) * dd_dr"),
    "self_block_transposed": ("Zblk[T + (size_t)S * ldz] = sb[T + (size_t)S * Nm];",
                              "Zblk[T + (size_t)S * ldz] = sb[S + (size_t)T * Nm];"),
    "grad_partner_sign": ("      grad[2 * n] -= gx;\n      grad[2 * n + 1] -= gy;",
                          "      grad[2 * n] += gx;\n      grad[2 * n + 1] += gy;"),
    "objective_not_modulus": ("J += creal(v) * creal(v) + cimag(v) * cimag(v);",
                              "J += creal(v) * creal(v) - cimag(v) * cimag(v);"),
    "transpose_solve_conjugated": ("for (int i = 0; i < k; ++i) s -= A[i + (size_t)k * lda] * b[i];",
                                   "for (int i = 0; i < k; ++i) s -= conj(A[i + (size_t)k * lda]) * b[i];"),
    "adjoint_contraction_transposed": ("G += Lam[i + (size_t)c * ld] * X[j + (size_t)c * ld];",
                                       "G += Lam[j + (size_t)c * ld] * X[i + (size_t)c * ld];"),
    "eep_phase_sign": ("s += c * Fj * cexp(I * ph);", "s += c * Fj * cexp(-I * ph);"),
    "eep_current_index_transposed": ("const cplx c = X[(size_t)i * Nm + j + (size_t)m * ldx];",
                                     "const cplx c = X[(size_t)j * Na + i + (size_t)m * ldx];"),
    "eep_pattern_conjugated": ("const cplx Fj = F[((size_t)comp * D + d) * Nm + j];",
                               "const cplx Fj = conj(F[((size_t)comp * D + d) * Nm + j]);"),
    "eep_uy_dropped": ("const double ph = k * (ux[d] * pos[2 * i] + uy[d] * pos[2 * i + 1]);",
                       "const double ph = k * (ux[d] * pos[2 * i]);"),
    "pattern_error_phi_dropped": ("eps[q] = sqrt(a * a + b * b) / norm;", "eps[q] = a / norm;"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique/found"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", str(mutated), "-o", str(lib), "-lm"])
    env = dict(os.environ, ORACLE_LIB=str(lib))
    # the pin file most likely to catch this mistake first (-x stops there)
    first = ("tests/test_oracle_grad.py" if name.startswith(("grad_", "adjoint_", "objective_"))
             else "tests/test_oracle_solve.py" if name.startswith(("lu_", "pivot_", "transpose_"))
             else "tests/test_oracle_eep.py" if name.startswith(("eep_", "pattern_"))
             else "tests/test_oracle_fill.py")
    pins = [first] + [f for f in PINS if f != first]
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutation {name}:\n{r.stdout[-2000:]}"
