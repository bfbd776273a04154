"""Planted mistakes in a copy of the oracle must be caught by the pins.

Each case rewrites one line of a private copy of qaoa_oracle.c (a dropped
term, a wrong sign, a wrong index, a transposed operand), compiles it into a
temporary directory, swaps it in for the real oracle and checks that at least
one pin check reports a large discrepancy. The real oracle is never touched.
"""
import os
import subprocess

import pytest

from oracle import oracle as O
from tests import oracle_pins as P

SRC = os.path.join(os.path.dirname(O.__file__), "qaoa_oracle.c")

MUTATIONS = {
    "mixer_sign": ("psi[x] = c * a - I * s * b;", "psi[x] = c * a + I * s * b;"),
    "mixer_transposed": ("psi[x | bit] = -I * s * a + c * b;", "psi[x | bit] = -I * s * b + c * a;"),
    "cost_sign": ("psi[x] *= cexp(-I * gamma * c);", "psi[x] *= cexp(I * gamma * c);"),
    "mixer_drops_last_qubit": ("for (int q = 0; q < n; q++)\n        oracle_apply_rx(n, q, beta, psi);",
                               "for (int q = 0; q < n - 1; q++)\n        oracle_apply_rx(n, q, beta, psi);"),
    "cut_wrong_index": ("uint64_t bv = (x >> edges[2 * e + 1]) & 1u;", "uint64_t bv = (x >> edges[2 * e]) & 1u;"),
    "layer_order": ("oracle_apply_cost(n, m, edges, gamma[l], psi);\n        oracle_apply_mixer(n, beta[l], psi);",
                    "oracle_apply_mixer(n, beta[l], psi);\n        oracle_apply_cost(n, m, edges, gamma[l], psi);"),
    "grad_beta_real_part": ("dbeta[l] = 2.0 * cimag(acc);", "dbeta[l] = 2.0 * creal(acc);"),
    "grad_gamma_dropped_factor": ("dgamma[l] = 2.0 * cimag(acc);", "dgamma[l] = cimag(acc);"),
    "grad_skips_undo_cost": ("oracle_apply_cost(n, m, edges, -gamma[l], lam);", ";"),
    "observable_weight_dropped": ("s += w[e];", "s += 1.0;"),
    "zz_sign": ("int sign = (((x >> u) ^ (x >> v)) & 1u) ? -1 : 1;", "int sign = (((x >> u) ^ (x >> v)) & 1u) ? 1 : -1;"),
    "plus_state_norm": ("double a = 1.0 / sqrt((double)N);", "double a = 1.0 / (double)N;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path, monkeypatch, oracle_lib):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mutated = tmp_path / "mutated.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "libmutated.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(mutated), "-lm"])
    monkeypatch.setattr(O, "_lib", O.load_library(str(so)))
    worst = {k: f() for k, f in P.ALL_CHECKS.items()}
    assert max(worst.values()) > 1e-3, worst
