"""Adjoint of the hit loop (fcs_simulate_backward) against the oracle's FP64
gradient and against FP64 central differences of the reweighted forward.

Bars: every gradient component within 1e-5 of the sum of the absolute values
of its terms (the oracle's gradient for |dL/dE_cell|) plus FP32 rounding of
the value: the GPU sums FP32 products E_hit dL/dE_cell over at most one warp
before its FP64 atomics, which bounds its error near 2e-6 of that sum; and
central differences (step 1e-4 of the parameter) within 1e-3 relative.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2103_14737_gb300 import fcs, synth  # noqa: E402
from paper_2103_14737_gb300.autograd import simulate_cells  # noqa: E402
from parity import check_grad, grad_scales  # noqa: E402

@pytest.fixture(scope="module")
def sim(geo, prm):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = fcs.Simulator(geo, prm)
    yield s
    s.close()


@pytest.mark.parametrize("case", ["electron", "ttbar", "ttbar_perevent"])
def test_backward_vs_oracle(sim, ogeo, oprm, prm, case):
    if case == "electron":
        parts, seed = synth.single_particle(3), 7
    else:
        parts, seed = synth.ttbar_like(2, 2), 11
    rng = np.random.default_rng(5)
    g = rng.normal(size=(parts.n_events, sim.n_cells)).astype(np.float32)
    d = sim.to_device(parts)
    r = sim.backward(d, seed, torch.as_tensor(g, device="cuda"), batched=0 if case == "ttbar_perevent" else 1)
    torch.cuda.synchronize()
    ref_f, ref_w = O.backward(ogeo, oprm, parts, seed, g.astype(np.float64))
    sc_f, sc_w = grad_scales(ogeo, oprm, prm, parts, seed, g.astype(np.float64))
    ref = O.simulate(ogeo, oprm, parts, seed, canon=False, cells64=False)
    assert r["stats"]["n_hits"] == ref.n_hits and r["stats"]["n_tasks"] == ref.n_tasks
    check_grad(r["d_frac"], r["d_shape_w"], ref_f, ref_w, sc_f, sc_w)


def test_backward_energy_interpolation(sim, ogeo, prm):
    """The adjoint with interpolated energy bins follows the forward's entries."""
    oprm_i = O.OracleParams(prm, energy_interp=1)
    parts, seed = synth.ttbar_like(6, 2, n=100), 13
    rng = np.random.default_rng(8)
    g = rng.normal(size=(parts.n_events, sim.n_cells)).astype(np.float32)
    r = sim.backward(sim.to_device(parts), seed, torch.as_tensor(g, device="cuda"), energy_interp=1)
    torch.cuda.synchronize()
    ref_f, ref_w = O.backward(ogeo, oprm_i, parts, seed, g.astype(np.float64))
    sc_f, sc_w = grad_scales(ogeo, oprm_i, prm, parts, seed, g.astype(np.float64))
    check_grad(r["d_frac"], r["d_shape_w"], ref_f, ref_w, sc_f, sc_w)


def test_backward_accumulates_and_offsets(sim, ogeo, oprm, prm):
    """Outputs accumulate; first_event selects the random streams."""
    parts, seed, fe = synth.ttbar_like(4, 1), 3, 1000
    g = np.ones((1, sim.n_cells), dtype=np.float32)
    d = sim.to_device(parts)
    gt = torch.as_tensor(g, device="cuda")
    r = sim.backward(d, seed, gt, first_event=fe)
    sim.backward(d, seed, gt, first_event=fe, d_frac=r["d_frac"], d_shape_w=r["d_shape_w"])
    torch.cuda.synchronize()
    ref_f, ref_w = O.backward(ogeo, oprm, parts, seed, g.astype(np.float64), first_event=fe)
    sc_f, sc_w = grad_scales(ogeo, oprm, prm, parts, seed, g.astype(np.float64), first_event=fe)
    check_grad(r["d_frac"] / 2, r["d_shape_w"] / 2, ref_f, ref_w, sc_f, sc_w)


def test_backward_ttbar_x32_central_differences(sim, ogeo, oprm, prm):
    """A 400-particle ttbar-like event simulated with 32 random streams;
    targets from layer fractions moved by +-10 %; quadratic loss."""
    parts, seed = synth.replicate(synth.ttbar_like(1, 1), 32), 1
    rng = np.random.default_rng(11)
    prm_t = dataclasses.replace(prm, frac=(prm.frac * rng.choice([0.9, 1.1], size=prm.frac.shape)).astype(np.float32))
    target = O.simulate(ogeo, O.OracleParams(prm_t), parts, seed, canon=False, tasks=False).cells64
    d = sim.to_device(parts)
    cells = sim.simulate(d, seed, dense=True)["cells"]
    g32 = (cells - torch.as_tensor(target, dtype=torch.float32, device="cuda")).contiguous()
    r = sim.backward(d, seed, g32)
    torch.cuda.synchronize()
    g = g32.cpu().numpy().astype(np.float64)
    ref_f, ref_w = O.backward(ogeo, oprm, parts, seed, g)
    sc_f, sc_w = grad_scales(ogeo, oprm, prm, parts, seed, g)
    check_grad(r["d_frac"], r["d_shape_w"], ref_f, ref_w, sc_f, sc_w)
    # central differences of the FP64 reweighted forward on 4 of the 32 streams
    sub = parts.events(0, 4)
    g_sub = sim.backward(sim.to_device(sub), seed, g32[:4].contiguous())
    torch.cuda.synchronize()
    gf = g_sub["d_frac"].cpu().numpy()
    gw = g_sub["d_shape_w"].cpu().numpy().reshape(-1, 128)
    tgt = target[:4]

    def loss(x):
        return 0.5 * ((x - tgt) ** 2).sum()

    # the FP64 cells of the loss: the oracle's reweighted forward at the base point
    base = O.reweighted_cells(ogeo, oprm, sub, seed)
    assert np.abs(base - cells[:4].cpu().numpy()).max() <= 1e-3 + 1e-5 * np.abs(base).max()
    f = prm.frac.reshape(-1).astype(np.float64)
    w = prm.shape_w.reshape(-1, 128).astype(np.float64)
    top = np.argsort(-np.abs(gf))[:3]
    for e in top:
        h = 1e-4 * f[e]
        fd = (loss(O.reweighted_cells(ogeo, oprm, sub, seed, f_entry=int(e), f_delta=h)) -
              loss(O.reweighted_cells(ogeo, oprm, sub, seed, f_entry=int(e), f_delta=-h))) / (2 * h)
        assert abs(gf[e] - fd) <= 1e-3 * abs(fd), (e, gf[e], fd)
    e = int(top[0])
    for b in np.argsort(-np.abs(gw[e]))[:3]:
        h = 1e-4 * w[e, b]
        fd = (loss(O.reweighted_cells(ogeo, oprm, sub, seed, w_entry=e, w_bin=int(b), w_delta=h)) -
              loss(O.reweighted_cells(ogeo, oprm, sub, seed, w_entry=e, w_bin=int(b), w_delta=-h))) / (2 * h)
        assert abs(gw[e, b] - fd) <= 1e-3 * abs(fd), (e, b, gw[e, b], fd)


def test_autograd_and_update(geo, prm, ogeo):
    """torch.autograd over the simulation; a gradient step pushed with
    fcs_update_params changes the forward exactly as the oracle with the new
    tables; an invalid update is refused and changes nothing."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = fcs.Simulator(geo, prm)  # its own tables: this test changes them
    try:
        parts, seed = synth.ttbar_like(3, 1), 2
        d = s.to_device(parts)
        frac = torch.tensor(prm.frac, device="cuda", requires_grad=True)
        w = torch.tensor(prm.shape_w, device="cuda", requires_grad=True)
        cells = simulate_cells(s, frac, w, d, seed)
        target = cells.detach() * 1.1
        loss = 0.5 * ((cells - target) ** 2).sum()
        loss.backward()
        direct = s.backward(d, seed, (cells - target).detach())
        torch.cuda.synchronize()
        torch.testing.assert_close(frac.grad.reshape(-1), direct["d_frac"], rtol=1e-5, atol=1e-3)
        torch.testing.assert_close(w.grad.reshape(-1), direct["d_shape_w"], rtol=1e-5, atol=1e-3)
        # a step on the fractions (kept >= 0), then the forward with the new tables
        with torch.no_grad():
            frac -= 1e-9 * frac.grad
            frac.clamp_(min=0.0)
        cells2 = simulate_cells(s, frac, w, d, seed).detach()
        prm2 = dataclasses.replace(prm, frac=frac.detach().cpu().numpy())
        ref = O.simulate(ogeo, O.OracleParams(prm2), parts, seed)
        det = s.simulate(d, seed, mode=fcs.MODE_DETERMINISTIC, dense=True)["cells"]
        assert np.array_equal(det.cpu().numpy().view(np.uint32), ref.cells_canon.view(np.uint32))
        err = np.abs(cells2.cpu().numpy() - ref.cells64)
        assert (err <= 1e-5 * np.abs(ref.cells64) + 1e-3).all()
        # invalid: a negative weight
        bad = w.detach().clone().reshape(-1)
        bad[5] = -1.0
        with pytest.raises(fcs.FcsError):
            s.update_params(shape_w=bad)
        det2 = s.simulate(d, seed, mode=fcs.MODE_DETERMINISTIC, dense=True)["cells"]
        assert torch.equal(det, det2)
    finally:
        s.close()
