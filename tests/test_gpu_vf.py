"""GPU volume fraction and its adjoint vs the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (Sigma - C) / T amplifies the field tolerance 1e-5 max(|Sigma|, C) by 1/T
# = 100 / C and the sigmoid's slope is at most 1/4: a sample moves by at most
# 2.5e-4 (at |Sigma| ~ C), so a cell mean does too.
VF_ATOL = 3e-4
GRAD_RTOL = 1e-4   # ||g_gpu - g_ref|| / ||g_ref||


@pytest.fixture(scope="module")
def c5():
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(5, small=True)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"])
    return cfg, lat


def _cells(cfg, **kw):
    c = dict(cfg["cells"])
    c.update(kw)
    return c


def test_vf_forward_parity(c5):
    from paper_2101_05031_gb300 import volume_fraction
    cfg, lat = c5
    cells = _cells(cfg)
    vf = volume_fraction(lat, cells).cpu().numpy().ravel()
    n = vf.size
    ids = np.random.default_rng(1).choice(n, 60, replace=False)
    ref = oracle.volume_fraction(cfg["nodes"], cfg["edges"], cfg["radius"], cells, R=cfg["R"],
                                 ids=ids)
    err = np.max(np.abs(vf[ids] - ref))
    assert err <= VF_ATOL, err
    assert np.all((vf >= 0) & (vf <= 1)) and vf.max() > 0.05


@pytest.mark.parametrize("m", [1, 2, 4])
def test_vf_forward_sample_counts(c5, m):
    from paper_2101_05031_gb300 import volume_fraction
    cfg, lat = c5
    cells = _cells(cfg, m=m)
    vf = volume_fraction(lat, cells).cpu().numpy().ravel()
    ids = np.random.default_rng(m).choice(vf.size, 40, replace=False)
    ref = oracle.volume_fraction(cfg["nodes"], cfg["edges"], cfg["radius"], cells, R=cfg["R"],
                                 ids=ids)
    assert np.max(np.abs(vf[ids] - ref)) <= VF_ATOL


def test_vf_hard_limit_isolated_strut():
    """T -> 0: the share of sample columns inside the circle of radius rho."""
    import paper_2101_05031_gb300 as cs
    from paper_2101_05031_gb300 import volume_fraction
    rho, R, m = 0.3, 0.45, 8
    lat = cs.Lattice(np.array([[0.5, 0.5, -5], [0.5, 0.5, 5]], np.float32), np.array([[0, 1]]),
                     np.array([rho], np.float32), R=R)
    cells = dict(origin=(0.0, 0.0, 0.0), h=1.0, dims=(1, 1, 1), m=m, T=1e-4)
    vf = float(volume_fraction(lat, cells).cpu()[0, 0, 0])
    k = (np.arange(m) + 0.5) / m
    X, Y = np.meshgrid(k, k)
    assert vf == pytest.approx(float(np.mean(np.hypot(X - 0.5, Y - 0.5) < rho)), abs=1e-6)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_vf_backward_parity(c5):
    from paper_2101_05031_gb300 import volume_fraction_backward
    cfg, lat = c5
    cells = _cells(cfg)
    dims = cells["dims"]
    n = dims[0] * dims[1] * dims[2]
    r = np.random.default_rng(2)
    ids = np.sort(r.choice(n, 40, replace=False))
    g = np.zeros(n, np.float32)
    g[ids] = r.normal(size=ids.size).astype(np.float32)
    gt = torch.from_numpy(g.reshape(dims[2], dims[1], dims[0])).cuda()
    gr, gn = volume_fraction_backward(lat, cells, gt)
    ref_r, ref_n = oracle.vf_backward(cfg["nodes"], cfg["edges"], cfg["radius"], cells,
                                      g[ids].astype(np.float64), R=cfg["R"], ids=ids)
    gr, gn = gr.cpu().numpy().astype(np.float64), gn.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(ref_r) > 0 and np.linalg.norm(ref_n) > 0
    er, en = _rel(gr, ref_r), _rel(gn, ref_n)
    assert er <= GRAD_RTOL, er
    assert en <= GRAD_RTOL, en
    # on 1000 (here: all touched) struts one by one, relative to the largest entry
    big = np.abs(ref_r) > 1e-3 * np.abs(ref_r).max()
    assert np.max(np.abs(gr - ref_r)[big] / np.abs(ref_r)[big]) < 1e-2


def test_vf_backward_deterministic(c5):
    from paper_2101_05031_gb300 import volume_fraction_backward
    cfg, lat = c5
    cells = _cells(cfg)
    d = cells["dims"]
    g = torch.randn((d[2], d[1], d[0]), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    a = volume_fraction_backward(lat, cells, g)
    b = volume_fraction_backward(lat, cells, g)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_autograd_function_and_radius_tuning():
    """The autograd.Function gives the same gradients, and a few gradient
    steps on the radii lower 1/2 ||vf - rho_target||^2."""
    import paper_2101_05031_gb300 as cs
    from paper_2101_05031_gb300 import VolumeFraction, volume_fraction_backward
    cfg = synth.config(5, small=True)
    cells = cfg["cells"]
    R = cfg["R"]
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=R)
    radius = torch.tensor(cfg["radius"], device="cuda", requires_grad=True)
    nodes = torch.tensor(cfg["nodes"], device="cuda", requires_grad=True)
    d = cells["dims"]
    o, h = cells["origin"], cells["h"]
    xs = o[0] + h * (torch.arange(d[0], device="cuda") + 0.5)
    ys = o[1] + h * (torch.arange(d[1], device="cuda") + 0.5)
    target = synth.graded_density(xs[None, None, :].double().cpu().numpy(),
                                  ys[None, :, None].double().cpu().numpy())
    target = torch.tensor(np.broadcast_to(target, (d[2], d[1], d[0])).copy(),
                          dtype=torch.float32, device="cuda")
    vf = VolumeFraction.apply(radius, nodes, lat, cells)
    loss = 0.5 * ((vf - target) ** 2).sum()
    loss.backward()
    gr, gn = volume_fraction_backward(lat, cells, (vf - target).detach())
    assert torch.allclose(radius.grad, gr, rtol=1e-6, atol=1e-12)
    assert torch.allclose(nodes.grad, gn, rtol=1e-6, atol=1e-12)
    losses = [float(loss.detach())]
    with torch.no_grad():
        r = radius.detach().clone()
    lr = 0.05 / max(float(gr.abs().max()), 1e-12)
    for _ in range(5):
        r.requires_grad_(True)
        vf = VolumeFraction.apply(r, nodes.detach(), lat, cells)
        loss = 0.5 * ((vf - target) ** 2).sum()
        loss.backward()
        with torch.no_grad():
            r = (r - lr * r.grad).clamp(0.05, 0.9 * R)
        losses.append(float(loss.detach()))
    assert losses[-1] < losses[0]


def test_cells_beyond_every_strut_support(c5):
    """Cells farther than R from every strut: Sigma = 0 at every sample, so
    each cell's volume fraction is sigma(-C/T) (below 1e-30 at T = 0.01 C) and
    no strut or node receives any gradient."""
    from paper_2101_05031_gb300 import volume_fraction, volume_fraction_backward
    cfg, lat = c5
    lo, hi = synth.lattice_bbox(cfg["nodes"])
    cells = dict(origin=(float(hi[0]) + 5.0, float(lo[1]), float(lo[2])), h=1.0, dims=(4, 3, 2),
                 m=2, T=0.01)
    vf = volume_fraction(lat, cells)
    assert vf.shape == (2, 3, 4)
    assert float(vf.abs().max()) <= 1e-30
    gr, gn = volume_fraction_backward(lat, cells, torch.ones((2, 3, 4), device="cuda"))
    assert int(torch.count_nonzero(gr)) == 0 and int(torch.count_nonzero(gn)) == 0
