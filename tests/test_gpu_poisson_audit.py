"""The FP32 Poisson path against the FP64 definition on millions of draws.

A hit count is n = Poisson(mu) (Listing 1, get_number_of_hits): inversion by
sequential search below mu = 10, PTRS (Hoermann 1993) above.  The library
draws it in FP32 wherever every comparison clears an error bound and in FP64,
the definition, where one does not.  The FP64 definition equals the oracle
draw for draw (the parity tests); this audit runs far more draws than the
oracle can and checks that each FP32 count the bounds certified is the
definition's count, and that few draws need FP64."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2103_14737_gb300 import fcs  # noqa: E402


@pytest.fixture(scope="module")
def sim(geo, prm):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = fcs.Simulator(geo, prm)
    yield s
    s.close()


def _means(seed, n):
    """Log-uniform means over [1e-3, 4096] (both methods, the FP32 range of
    PTRS), plus means at the method boundary: the floats just below 10 and 10
    itself."""
    rng = np.random.default_rng(seed)
    mu = np.exp(rng.uniform(np.log(1e-3), np.log(4096.0), n)).astype(np.float32)
    below = np.nextafter(np.float32(10.0), np.float32(0.0))
    mu[: n // 64] = below
    mu[n // 64: n // 32] = np.float32(10.0)
    return mu


@pytest.mark.parametrize("seed", [3, 11])
def test_certified_fp32_counts_equal_the_definition(sim, seed):
    n = 1 << 23
    mu = _means(seed, n)
    n32, n64 = fcs.fcs_poisson_audit(sim.prm, torch.from_numpy(mu).cuda(), seed=0x5EED0000 + seed)
    torch.cuda.synchronize()
    a = n32.cpu().numpy().astype(np.int64)
    b = n64.cpu().numpy().astype(np.int64)
    cert = a >= 0
    bad = np.flatnonzero(cert & (a != b))
    assert bad.size == 0, f"{bad.size} certified FP32 counts differ, e.g. mu={mu[bad[:5]]} fp32={a[bad[:5]]} fp64={b[bad[:5]]}"
    inv = mu < 10.0
    mid = ~inv & (mu < 300.0)
    # the uncertain share the error bounds leave: about 1e-4 of the
    # inversions, a few 1e-4 of the PTRS draws below mu = 300 (most pile-up
    # draws) and a few 1e-3 over the whole FP32 range
    assert (~cert[inv]).mean() < 3e-4
    assert (~cert[mid]).mean() < 2e-3
    assert (~cert[~inv]).mean() < 2e-2
    print("uncertain: inversion %.2e, PTRS below 300 %.2e, PTRS %.2e"
          % ((~cert[inv]).mean(), (~cert[mid]).mean(), (~cert[~inv]).mean()))
    # the definition's counts have the Poisson mean (loose: 8 sigma of the
    # sample mean of all counts)
    assert abs(b.mean() - mu.astype(np.float64).mean()) < 8 * np.sqrt(mu.astype(np.float64).mean() / n)
