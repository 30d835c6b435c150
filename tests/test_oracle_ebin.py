"""Pins of the probabilistic energy-bin interpolation (an option of the
parametrisation selection): E = m 2^k, m in [1, 2), takes the next energy
bin with probability m - 1, decided by u = x0 2^-32 of Philox block
(0, 2 << 16, particle in event, event) < m - 1."""
import numpy as np
import pytest

from oracle import oracle as O


@pytest.fixture(scope="module")
def oprm_i(prm):
    return O.OracleParams(prm, energy_interp=1)


def _bins(prm, entry):
    NE, NH = prm.frac.shape[1], prm.frac.shape[2]
    return (entry // NH) % NE


def test_off_is_plain_selection(oprm, prm):
    rng = np.random.default_rng(1)
    for _ in range(200):
        t, E, eta = int(rng.integers(0, 3)), float(np.float32(2.0 ** rng.uniform(5, 23))), float(rng.uniform(-5, 5))
        assert O.param_entry_rng(oprm, t, E, eta, 7, 3, 11) == O.param_entry(oprm, t, E, eta)


def test_integer_rule(oprm, oprm_i, prm):
    """The choice equals x0 < mantissa23 << 9 with x0 from the pinned Philox."""
    rng = np.random.default_rng(2)
    NE = prm.frac.shape[1]
    seed = 0x1234_5678_9ABC
    n_up = 0
    for i in range(400):
        E = np.float32(2.0 ** rng.uniform(6, 22))
        t, eta, p, ev = int(rng.integers(0, 3)), float(rng.uniform(-3, 3)), int(rng.integers(0, 5000)), i
        base = O.param_entry(oprm, t, float(E), eta)
        got = O.param_entry_rng(oprm_i, t, float(E), eta, seed, p, ev)
        x0 = int(O.philox(np.array([[0, 2 << 16, p, ev]], dtype=np.uint32), seed)[0, 0])
        mant = int(E.view(np.uint32)) & 0x7FFFFF
        up = x0 < (mant << 9)
        eb = _bins(prm, base)
        want_eb = min(eb + 1, NE - 1) if up else eb
        assert _bins(prm, got) == want_eb, (E, x0, mant)
        assert got - base == (want_eb - eb) * prm.frac.shape[2]
        n_up += up
    assert 100 < n_up < 300


def test_fraction_and_edges(oprm, oprm_i, prm):
    NE = prm.frac.shape[1]
    # m - 1 = 0.25: a quarter of the particles take the next bin
    E = float(1.25 * 2.0 ** 12)
    base = O.param_entry(oprm, 0, E, 0.3)
    ups = sum(O.param_entry_rng(oprm_i, 0, E, 0.3, 99, p, 5) != base for p in range(20000))
    z = (ups - 5000) / np.sqrt(20000 * 0.25 * 0.75)
    assert abs(z) < 4.5, z
    # a power of two never moves; the last bin stays the last bin
    E2 = float(2.0 ** 12)
    assert all(O.param_entry_rng(oprm_i, 1, E2, 1.0, 3, p, 0) == O.param_entry(oprm, 1, E2, 1.0) for p in range(500))
    Etop = float(1.9 * 2.0 ** (prm.ebin_log2_min + NE - 1))
    top = O.param_entry(oprm, 2, Etop, 2.0)
    assert _bins(prm, top) == NE - 1
    assert all(O.param_entry_rng(oprm_i, 2, Etop, 2.0, 3, p, 0) == top for p in range(200))
    # below the table: the points 2^k and 2^(k+1) of E = 1.75 2^k with k + 1 <= ebin_log2_min both
    # clamp to bin 0, so the particle never moves; from 2^ebin_log2_min on it moves to bin 1
    for k in (prm.ebin_log2_min - 3, prm.ebin_log2_min - 1):
        Elow = float(1.75 * 2.0 ** k)
        low = O.param_entry(oprm, 0, Elow, 0.4)
        assert _bins(prm, low) == 0
        assert all(O.param_entry_rng(oprm_i, 0, Elow, 0.4, 3, p, 1) == low for p in range(300))
    E0 = float(1.75 * 2.0 ** prm.ebin_log2_min)
    moved = {_bins(prm, O.param_entry_rng(oprm_i, 0, E0, 0.4, 3, p, 1)) for p in range(300)}
    assert moved == {0, 1}


def test_simulation_uses_interpolated_entries(ogeo, oprm, oprm_i, prm):
    from paper_2103_14737_gb300 import synth
    parts = synth.ttbar_like(5, 2, n=60)
    a = O.simulate(ogeo, oprm, parts, 4)
    b = O.simulate(ogeo, oprm_i, parts, 4)
    assert a.n_tasks > 0 and b.n_tasks > 0
    # same particles, some in the next energy bin: the totals differ, both conserve
    assert not np.array_equal(a.cells64, b.cells64)
    np.testing.assert_allclose(b.cells64.sum(), b.E_layers, rtol=1e-6)
