"""Free-field dispersion relations on the GPU (bri_dispersion, Sec. 2 / App. A)
against the oracle's solver, which is pinned by the paper's closed forms and
expansions: Wilson and Brillouin kernels and their overlaps, masses 0 to 0.75,
momenta along the three lattice directions the paper plots and off-axis."""
import numpy as np
import pytest

from oracle import dispersion as odisp
from paper_1701_00726_gb300 import KERNEL_BRILLOUIN, KERNEL_WILSON, dispersion

pytestmark = pytest.mark.gpu


def _points():
    pts = []
    for direction in ((1, 0, 0), (1, 1, 0), (1, 1, 1), (0.9, 0.5, -0.3)):
        for t in (0.0, 0.2, 0.7, 1.5, 2.8):
            for am in (0.0, 0.05, 0.75):
                pts.append((tuple(t * np.array(direction, dtype=float)), am))
    return pts


@pytest.mark.parametrize("kernel", ["wil", "bri"])
@pytest.mark.parametrize("overlap,rho", [(False, 1.0), (True, 1.0), (True, (3 - 3 ** 0.5) / 2)])
def test_dispersion_vs_oracle(kernel, overlap, rho):
    pts = _points()
    got = dispersion([p for p, _ in pts], [m for _, m in pts],
                     kernel=KERNEL_BRILLOUIN if kernel == "bri" else KERNEL_WILSON, overlap=overlap, rho=rho)
    for (p, am), e in zip(pts, got):
        want = odisp.energy(p, am, kernel, overlap=overlap, rho=rho)
        if np.isnan(want):
            assert np.isnan(e), (p, am)
        else:
            assert abs(e - want) <= 1e-12 * max(1.0, want), (p, am, e, want)
