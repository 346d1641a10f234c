"""The seeded input generators (qcs_inputs) hold no arithmetic of the method,
but the circuits they draw must be the gates they claim to be."""
import numpy as np

import qcs_inputs as qi


def test_fsim_quarter_turn_has_exact_zeros():
    """fSim(pi/2, phi): cos(pi/2) = 0 exactly, so the gate has exactly four
    nonzero entries -- not 6e-17, the rounding error of the double nearest
    pi/2, which would spread tiny nonzeros through a network."""
    g = qi.fsim(np.pi / 2, np.pi / 6)
    assert g[1, 1] == 0 and g[2, 2] == 0
    assert np.count_nonzero(g) == 4
    assert np.count_nonzero(g.astype(np.complex64)) == 4
    assert np.allclose(g.conj().T @ g, np.eye(4), atol=1e-15)
    assert qi.fsim(np.pi, 0.3)[1, 2] == 0 and qi.fsim(-np.pi / 2, 0.3)[1, 1] == 0


def test_fsim_entries_match_cos_and_sin():
    rng = np.random.default_rng(0)
    for th in np.concatenate([rng.uniform(-np.pi, np.pi, 200), [0.0, np.pi / 4, 3 * np.pi / 4]]):
        ph = float(rng.uniform(0, np.pi))
        g = qi.fsim(th, ph)
        assert abs(g[1, 1].real - np.cos(th)) <= 4e-16
        assert abs(-g[1, 2].imag - np.sin(th)) <= 4e-16
        assert np.allclose(g.conj().T @ g, np.eye(4), atol=1e-15)
        assert g[3, 3] == np.exp(-1j * ph)


def test_grid_circuit_fsim_gates_are_exactly_sparse():
    circ = qi.random_grid_circuit(3, 4, 8, seed=0)
    fs = [g for g in circ.gates if g.name == "fsim"]
    assert fs and all(np.count_nonzero(g.matrix.astype(np.complex64)) == 4 for g in fs)
