"""The CPU oracle against values fixed by the paper and by mathematics.

Tolerances: the oracle is FP64 throughout, so every pin that compares two
FP64 computations of the same exact quantity allows 1e-11 (relative to
max(|value|, 1)); the finite-difference pin allows 1e-6 because central
differences with h = 1e-5 carry O(h^2) truncation error.
"""
import numpy as np
import pytest

from tests import oracle_pins as P
from oracle import oracle as O
from paper_2410_22247_gb300 import workloads as W


def test_oracle_matches_dense_matrix_exponentials(oracle_lib):
    assert P.check_bruteforce() < 1e-12


def test_oracle_matches_published_p1_closed_form(oracle_lib):
    assert P.check_closed_form() < 1e-11


def test_oracle_matches_symmetric_subspace_models(oracle_lib):
    assert P.check_symmetric() < 1e-11


def test_adjoint_gradient_matches_finite_differences(oracle_lib):
    assert P.check_finite_difference() < 1e-6


def test_oracle_invariants(oracle_lib):
    assert P.check_invariants() < 1e-11


def test_complete_graph_k12_reference_point(oracle_lib):
    # K_12, p = 1, gamma = 0.4, beta = 0.3: closed form and Dicke model agree
    from oracle import closed_form as CF, symmetric as SYM
    n, e = W.complete_graph(12)
    E = O.energy(n, e, [0.4], [0.3])
    assert abs(E - CF.energy_p1(n, e, 0.4, 0.3)) < 1e-11 * E
    assert abs(E - SYM.energy(SYM.complete_graph_model(12), [0.4], [0.3])) < 1e-11 * E


def test_cut_value_by_hand(oracle_lib):
    # path 0-1-2: x = 0b010 cuts both edges, x = 0b011 cuts one
    e = W.canonical_edges([(0, 1), (1, 2)])
    assert O.cut_value(e, 0b010) == 2
    assert O.cut_value(e, 0b011) == 1
    assert O.cut_value(e, 0b000) == 0
    obs = (W.canonical_edges([(0, 2)]), np.array([5.0]))
    assert O.observable_value(obs, 0b001) == 5.0
    assert O.observable_value(obs, 0b101) == 0.0


def test_single_qubit_rx_by_hand(oracle_lib):
    # RX(2b)|0> = cos b |0> - i sin b |1>
    psi = np.array([1.0, 0.0], dtype=np.complex128)
    O.apply_rx(1, 0, 0.3, psi)
    assert np.allclose(psi, [np.cos(0.3), -1j * np.sin(0.3)], atol=1e-15)


def test_max_cut_closed_forms(oracle_lib):
    """Tree, K_n, cycle, K_{a,b} and Petersen maxima and the smallest
    maximiser (oracle_pins.check_max_cut)."""
    assert P.check_max_cut() == 0


def test_inverse_cdf_sampler(oracle_lib):
    """Basis state, |+>^n and stratified uniforms on a random state
    (oracle_pins.check_sampler)."""
    assert P.check_sampler() == 0


def test_weighted_oracle_matches_dense_and_scaling(oracle_lib):
    assert P.check_weighted() < 1e-11


def test_weighted_max_cut_pins(oracle_lib):
    # uniform weight c scales every cut by c; a path with weights (1, 5, 1)
    # cuts all three edges (bipartite)
    n, e = W.cycle_graph(7)
    assert O.max_cut_w(n, e, [3] * 7)[0] == 3 * O.max_cut(n, e)[0]
    path = W.canonical_edges([(0, 1), (1, 2), (2, 3)])
    assert O.max_cut_w(4, path, [1, 5, 1])[0] == 7
    # triangle with weights (1, 2, 3): the best cut leaves out the lightest edge
    tri = W.canonical_edges([(0, 1), (0, 2), (1, 2)])
    assert O.max_cut_w(3, tri, [1, 2, 3])[0] == 5


def test_lightcone_matches_full_statevector(oracle_lib):
    """oracle/lightcone.py (per-edge reverse causal cones, Sec. 5.1) against
    the full C oracle: energy and every gradient component of H_C and of a
    weighted edge subset, to 1e-11, on graphs whose radius-p balls leave
    vertices out (cycle, 3-regular, path, caterpillar) and on a star, whose
    ball is the whole graph."""
    assert P.lightcone_cases_leave_vertices_out() >= 8
    assert P.check_lightcone() < 1e-11


def test_ising_oracle_matches_dense_exponentials(oracle_lib):
    """Real weights of both signs and real fields: the Ising-form oracle's
    state against expm of the dense H and H_M, amplitude by amplitude."""
    assert P.check_ising_dense() < 1e-12


def test_ising_oracle_fields_only_closed_form(oracle_lib):
    """No edges, p = 1: E = sum_i h_i/2 (1 + sin 2 beta sin gamma h_i) and its
    derivatives (independent qubits)."""
    assert P.check_ising_fields_closed_form() < 1e-12


def test_ising_oracle_reduces_to_maxcut_and_weighted_maxcut(oracle_lib):
    assert P.check_ising_reductions() < 1e-11


def test_ising_oracle_gradient_matches_finite_differences(oracle_lib):
    assert P.check_ising_finite_difference() < 1e-6


def test_ising_oracle_invariants_under_weight_and_field_preserving_automorphisms(oracle_lib):
    assert P.check_ising_invariants() < 1e-11


def test_ising_lightcone_matches_full_statevector(oracle_lib):
    """Per-term light cones (ZZ terms and field terms) of Ising objectives
    against the full Ising oracle, to 1e-11."""
    assert P.check_ising_lightcone() < 1e-11
