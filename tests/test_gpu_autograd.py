"""torch.autograd over the discrete adjoint: gradients flow to tau and the
inlet amplitudes and agree with central differences of the FP64 forward."""
import numpy as np
import pytest
import torch

from paper_2202_11770_gb300 import geometry as geo

pytestmark = pytest.mark.gpu
hemegb = pytest.importorskip("paper_2202_11770_gb300.hemegb")
adjoint = pytest.importorskip("paper_2202_11770_gb300.adjoint")


def test_autograd_matches_finite_differences():
    lat = geo.tree(1, 7, root_radius=4.0, length_ratio=5.0, n_sectors=2, n_rings=2)
    s = hemegb.Solver(lat, tau=0.7, precision="fp64")
    for k in range(1, len(lat.iolets)):
        s.set_pressure(k, 1.0)
    sites = np.nonzero(lat.xyz[:, 2] == int(lat.info["root_length"] // 2))[0]
    target = np.full(sites.size, 0.02)
    waves = {0: {"kind": "cosine", "mean": 0.03, "rel": 0.5, "period": 50.0}}
    N = 40
    tau = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
    amps = torch.tensor([1.0, 0.9, 1.1, 0.95], dtype=torch.float64, requires_grad=True)
    J = adjoint.flow_objective(tau, amps, s, N, sites, target, [0, 0, 1], waves)
    (3.0 * J).backward()
    h = 1e-5

    def run(t, a):
        with torch.no_grad():
            return float(adjoint.flow_objective(torch.tensor(t, dtype=torch.float64),
                                                torch.tensor(a, dtype=torch.float64), s, N, sites, target,
                                                [0, 0, 1], waves))
    fd = (run(0.7 + h, amps.detach().numpy()) - run(0.7 - h, amps.detach().numpy())) / (2 * h)
    assert tau.grad.item() == pytest.approx(3.0 * fd, rel=1e-6)
    for g in range(4):
        e = np.zeros(4)
        e[g] = h
        a = amps.detach().numpy()
        fd = (run(0.7, a + e) - run(0.7, a - e)) / (2 * h)
        assert amps.grad[g].item() == pytest.approx(3.0 * fd, rel=1e-6)
