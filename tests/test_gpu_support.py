"""Self-support metrics on the GPU (csl_support_metrics) against the reference."""
import numpy as np
import pytest

import synth
from oracle import support

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("idx", [1, 2, 3])
def test_support_metrics_match_reference(idx):
    import paper_2101_05031_gb300 as cs
    cfg = synth.config(idx, small=True)
    lat = cs.Lattice(cfg["nodes"], cfg["edges"], cfg["radius"], R=cfg["R"], C=cfg["C"])
    for t_p, alpha in (((0, 0, 1), np.pi / 4), ((0.3, -0.2, 1.0), np.pi / 3), ((1, 0, 0), 0.5)):
        g, p = lat.support_metrics(t_p, alpha)
        rg, rp = support.support_metrics(cfg["nodes"], cfg["edges"], cfg["radius"], t_p, alpha)
        assert g == pytest.approx(rg, rel=1e-9, abs=1e-12)
        assert p == pytest.approx(rp, rel=1e-9, abs=1e-12)
    # deterministic
    assert lat.support_metrics() == lat.support_metrics()
    with pytest.raises(cs.CslError):
        lat.support_metrics((0, 0, 0))
