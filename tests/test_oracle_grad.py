"""Pins of the oracle's differentiable form (reweighted forward and gradient).

With the seed fixed, every hit keeps its task, count n, shape bin and cell;
a change of the layer fraction f moves each hit energy to E f / n and a
change of the shape weights multiplies it by the likelihood ratio
p_b(w) / p_b(w0), p_b = w_b / sum(w).  The pins are independent of the
gradient code: the reweighted forward against the hit dump of the plain
simulation, closed forms (a loss linear in the cells, invariance of the
shape under a common scale of its weights) and FP64 central differences.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_14737_gb300 import synth

SEED = 5


@pytest.fixture(scope="module")
def case(ogeo, oprm, prm):
    parts = synth.single_particle(2, E=32768.0, eta=0.6)
    r = O.simulate(ogeo, oprm, parts, SEED, hit_cap=20000)
    assert r.n_hits < 20000
    base = np.array([O.param_entry(oprm, int(t), float(E), float(eta))
                     for t, E, eta in zip(parts.type, parts.E, parts.eta)])
    NL = prm.frac.shape[-1]
    # per-hit FP64 energy E f / n and the entry of its task, from the dumps
    tp = parts.event_offsets[r.task_event] + r.task_particle
    t_entry = base[tp] * NL + r.task_layer
    t_E = parts.E[tp].astype(np.float64)
    t_f = prm.frac.reshape(-1)[t_entry].astype(np.float64)
    t_e64 = t_E * t_f / r.task_n
    hit_task = np.repeat(np.arange(r.n_tasks), r.task_n[:r.n_tasks])
    return dict(parts=parts, r=r, t_entry=t_entry, t_E=t_E, t_n=r.task_n[:r.n_tasks].astype(np.float64),
                t_e64=t_e64, hit_task=hit_task, hit_ev=r.task_event[hit_task],
                hit_cell=r.hit_cell[:r.n_hits], hit_bin=r.hit_bin[:r.n_hits].astype(np.int64))


def _cells_from_hits(c, ogeo, e_hit):
    out = np.zeros((len(c["parts"].event_offsets) - 1, ogeo.n_cells))
    np.add.at(out, (c["hit_ev"], c["hit_cell"]), e_hit)
    return out


def test_reweighted_identity(case, ogeo, oprm):
    """No change: the FP64 hit energies of the plain simulation's hits."""
    c = case
    rw = O.reweighted_cells(ogeo, oprm, c["parts"], SEED)
    ref = _cells_from_hits(c, ogeo, c["t_e64"][c["hit_task"]])
    np.testing.assert_allclose(rw, ref, rtol=1e-13, atol=1e-9)
    # and the simulation's own FP64 cells, which sum fl32(E_l / n)
    np.testing.assert_allclose(rw, c["r"].cells64, rtol=2e-7, atol=1e-6)


def test_reweighted_frac_shift(case, ogeo, oprm, prm):
    c = case
    e = int(c["t_entry"][0])
    d = 0.01
    rw = O.reweighted_cells(ogeo, oprm, c["parts"], SEED, f_entry=e, f_delta=d)
    f = prm.frac.reshape(-1).astype(np.float64)
    fe = np.where(c["t_entry"] == e, f[c["t_entry"]] + d, f[c["t_entry"]])
    ref = _cells_from_hits(c, ogeo, (c["t_E"] * fe / c["t_n"])[c["hit_task"]])
    np.testing.assert_allclose(rw, ref, rtol=1e-13, atol=1e-9)


def test_reweighted_bin_doubling(case, ogeo, oprm, prm):
    """Doubling w_b scales bin b's hits by 2W/(W+w_b) and the others by W/(W+w_b)."""
    c = case
    e = int(c["t_entry"][0])
    sel = c["t_entry"][c["hit_task"]] == e
    b = int(np.bincount(c["hit_bin"][sel], minlength=128).argmax())
    w = prm.shape_w.reshape(-1, 128)[e].astype(np.float64)
    W = w.sum()
    rw = O.reweighted_cells(ogeo, oprm, c["parts"], SEED, w_entry=e, w_bin=b, w_delta=float(w[b]))
    scale = np.ones(c["r"].n_hits)
    scale[sel] = W / (W + w[b])
    scale[sel & (c["hit_bin"] == b)] = 2 * W / (W + w[b])
    ref = _cells_from_hits(c, ogeo, c["t_e64"][c["hit_task"]] * scale)
    np.testing.assert_allclose(rw, ref, rtol=1e-12, atol=1e-9)


def test_backward_linear_loss(case, ogeo, oprm, prm):
    """L = sum of all cells: dL/df[e] = sum over e's tasks of the particle energy."""
    c = case
    g = np.ones((2, ogeo.n_cells))
    d_frac, d_w = O.backward(ogeo, oprm, c["parts"], SEED, g)
    ref = np.zeros(prm.frac.size)
    np.add.at(ref, c["t_entry"], c["t_E"])
    np.testing.assert_allclose(d_frac, ref, rtol=1e-12, atol=0)
    # per bin: A_k = sum of the bin's hit energies, gradient A_k / w_k - sum(A) / W
    e = int(c["t_entry"][0])
    sel = c["t_entry"][c["hit_task"]] == e
    A = np.bincount(c["hit_bin"][sel], weights=c["t_e64"][c["hit_task"]][sel], minlength=128)
    w = prm.shape_w.reshape(-1, 128)[e].astype(np.float64)
    ref_w = np.where(w > 0, A / np.where(w > 0, w, 1), 0) - A.sum() / w.sum()
    np.testing.assert_allclose(d_w[e], ref_w, rtol=1e-10, atol=1e-9 * np.abs(ref_w).max())


def test_backward_scale_invariance(case, ogeo, oprm, prm):
    """p_b is unchanged by a common scale of w, so sum_k w_k dL/dw_k = 0."""
    c = case
    rng = np.random.default_rng(3)
    g = rng.normal(size=(2, ogeo.n_cells))
    _, d_w = O.backward(ogeo, oprm, c["parts"], SEED, g)
    w = prm.shape_w.reshape(-1, 128).astype(np.float64)
    for e in np.unique(c["t_entry"]):
        s = (w[e] * d_w[e]).sum()
        assert abs(s) <= 1e-10 * np.abs(w[e] * d_w[e]).sum() + 1e-300, (e, s)


def test_backward_central_differences(case, ogeo, oprm, prm):
    """Quadratic loss against targets from fractions moved by +-10 %: the
    analytic gradient equals FP64 central differences (step 1e-4, relative)."""
    c = case
    rng = np.random.default_rng(11)
    prm_t = dataclasses.replace(prm, frac=(prm.frac * rng.choice([0.9, 1.1], size=prm.frac.shape)
                                           ).astype(np.float32))
    target = O.simulate(ogeo, O.OracleParams(prm_t), c["parts"], SEED, canon=False, tasks=False).cells64
    cells = O.reweighted_cells(ogeo, oprm, c["parts"], SEED)

    def loss(x):
        return 0.5 * ((x - target) ** 2).sum()

    d_frac, d_w = O.backward(ogeo, oprm, c["parts"], SEED, cells - target)
    entries = np.unique(c["t_entry"])
    f = prm.frac.reshape(-1).astype(np.float64)
    for e in entries[:6]:
        h = 1e-4 * f[e]
        lp = loss(O.reweighted_cells(ogeo, oprm, c["parts"], SEED, f_entry=int(e), f_delta=h))
        lm = loss(O.reweighted_cells(ogeo, oprm, c["parts"], SEED, f_entry=int(e), f_delta=-h))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - d_frac[e]) <= 1e-3 * abs(fd) + 1e-9, (e, fd, d_frac[e])
    w = prm.shape_w.reshape(-1, 128).astype(np.float64)
    e = int(c["t_entry"][0])
    sel = c["t_entry"][c["hit_task"]] == e
    counts = np.bincount(c["hit_bin"][sel], minlength=128)
    hit_bins = list(np.argsort(-counts)[:4])
    empty = [k for k in range(128) if counts[k] == 0 and w[e, k] > 0][:2]
    assert empty, "want a bin with weight but no hits"
    for b in hit_bins + empty:
        h = 1e-4 * w[e, b]
        lp = loss(O.reweighted_cells(ogeo, oprm, c["parts"], SEED, w_entry=e, w_bin=int(b), w_delta=h))
        lm = loss(O.reweighted_cells(ogeo, oprm, c["parts"], SEED, w_entry=e, w_bin=int(b), w_delta=-h))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - d_w[e, b]) <= 1e-3 * abs(fd) + 1e-6 * np.abs(d_w[e]).max(), (b, fd, d_w[e, b])
