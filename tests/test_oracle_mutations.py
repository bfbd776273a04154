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
    "grad_beta_real_part": ("acc_im += cimag(conj(lam[x]) * phi[x ^ bit]);",
                            "acc_im += creal(conj(lam[x]) * phi[x ^ bit]);"),
    "grad_gamma_dropped_factor": ("dgamma[l] = 2.0 * acc_im;", "dgamma[l] = acc_im;"),
    "grad_skips_undo_cost": ("oracle_apply_cost(n, m, edges, -gamma[l], lam);", ";"),
    "observable_weight_dropped": ("s += w[e];", "s += 1.0;"),
    "zz_sign": ("int sign = (((x >> u) ^ (x >> v)) & 1u) ? -1 : 1;", "int sign = (((x >> u) ^ (x >> v)) & 1u) ? 1 : -1;"),
    "plus_state_norm": ("double a = 1.0 / sqrt((double)N);", "double a = 1.0 / (double)N;"),
    "ising_field_dropped": ("                s += h[i];", "                s += 0.0;"),
    "ising_field_on_wrong_value": ("if ((x >> i) & 1u)", "if (!((x >> i) & 1u))"),
    "ising_cost_sign": ("psi[x] *= cexp(-I * gamma * oracle_ising_value(m, edges, w, n, h, x));",
                        "psi[x] *= cexp(I * gamma * oracle_ising_value(m, edges, w, n, h, x));"),
    "ising_gamma_grad_uses_observable": (
        "im_sum += cimag(conj(lam[x]) * oracle_ising_value(m, edges, w, n, h, x) * phi[x]);",
        "im_sum += cimag(conj(lam[x]) * oracle_ising_value(k, oedges, ow, n, oh, x) * phi[x]);"),
    "terms_zz_sign": ("s += w[e] * 0.5 * (1.0 - oracle_zz(", "s += w[e] * 0.5 * (1.0 + oracle_zz("),
    "max_cut_comparison_flipped": ("if (c > best) {", "if (c < best) {"),
    "max_cut_ties_take_the_last": ("if (c > best) {", "if (c >= best) {"),
    "sampler_exclusive_cdf": ("        s += a * a + b * b;\n        cdf[x] = s;",
                              "        cdf[x] = s;\n        s += a * a + b * b;"),
    "sampler_unnormalised": ("const double t = u[k] * s;", "const double t = u[k];"),
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


# Planted mistakes in a copy of oracle/lightcone.py. Removing the edges whose
# two ends both lie at distance p is not among them: those edges cancel in the
# reverse causal cone (Sec. 5.1), and check_lightcone verifies that identity.
LC_SRC = os.path.join(os.path.dirname(O.__file__), "lightcone.py")
LC_MUTATIONS = {
    "ball_radius_p_minus_1": ("if dist[a] == p:", "if dist[a] == p - 1:"),
    "ball_grown_from_one_end": ("q = deque([u, v])", "q = deque([u])"),
    "observed_edge_left_out_of_the_cost": ("if int(a) in index and int(b) in index]",
                                           "if int(a) in index and int(b) in index and {int(a), int(b)} != {u, v}]"),
    "subset_weight_dropped": ("wk = w[e] if w is not None else float(weights[k])", "wk = 1.0"),
    "gradient_of_one_layer_dropped": ("dg += wk * dge", "dg[1:] += wk * dge[1:]"),
    "ising_cone_without_fields": ("fn = oracle.ising(sub, w[inside], np.array([h[a] for a in verts]))",
                                  "fn = oracle.ising(sub, w[inside], np.zeros(len(verts)))"),
    "ising_field_term_without_cone": ("        terms += [((i, i), None, h[i]) for i in range(n)]", "        pass"),
}


def _load_mutated_lightcone(src, tag):
    import types
    mod = types.ModuleType(f"oracle.lightcone_{tag}")
    mod.__dict__["__package__"] = "oracle"
    exec(compile(src, f"lightcone_{tag}.py", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(LC_MUTATIONS))
def test_lightcone_pin_catches_planted_mistake(name, oracle_lib):
    old, new = LC_MUTATIONS[name]
    src = open(LC_SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mutated = _load_mutated_lightcone(src.replace(old, new), name)
    worst = max(P.check_lightcone(mutated), P.check_ising_lightcone(mutated))
    assert worst > 1e-3, worst


def test_lightcone_unmutated_copy_passes(oracle_lib):
    assert P.check_lightcone(_load_mutated_lightcone(open(LC_SRC).read(), "copy")) < 1e-11


# Planted mistakes in a copy of oracle/oracle.py's integer-weight route
# (weighted MaxCut as the plain cut of the edge list in which edge e appears
# w_e times, with (edges, w) as the observable); the copy runs on the same
# compiled oracle.
OR_MUTATIONS = {
    "weighted_cost_ignores_weights": ("return _edges(np.repeat(e, w, axis=0))", "return _edges(e)"),
    "weighted_observable_unit_weights": ("return _edges(edges), _f64(weights)",
                                         "return _edges(edges), np.ones(len(_edges(edges)))"),
}


def _load_mutated_oracle(src, tag):
    import types
    mod = types.ModuleType(f"oracle.oracle_{tag}")
    mod.__dict__.update(__file__=O.__file__, __package__="oracle")
    exec(compile(src, f"oracle_{tag}.py", "exec"), mod.__dict__)
    mod._lib = O._load()
    return mod


@pytest.mark.parametrize("name", sorted(OR_MUTATIONS))
def test_weighted_pin_catches_planted_mistake(name, monkeypatch, oracle_lib):
    old, new = OR_MUTATIONS[name]
    src = open(O.__file__).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    monkeypatch.setattr(P, "O", _load_mutated_oracle(src.replace(old, new), name))
    worst = P.check_weighted()
    assert worst > 1e-3, worst


def test_weighted_unmutated_copy_passes(monkeypatch, oracle_lib):
    monkeypatch.setattr(P, "O", _load_mutated_oracle(open(O.__file__).read(), "copy"))
    assert P.check_weighted() < 1e-11
