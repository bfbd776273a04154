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
