"""Host-side observables of the planar sweeps (Sec. III), on CPU: the library's
density error, interface width and surface tension against the oracle's
independent implementations."""
import pytest

pytest.importorskip("paper_2107_06355_gb300")
import numpy as np

from oracle import lbm as OL
from paper_2107_06355_gb300 import sweeps as SW


def test_sweep_observables_match_oracle_definitions():
    """The sweep's host-side observables (density error, interface width, surface
    tension) agree with the oracle's independent implementations on seeded profiles."""
    rng = np.random.default_rng(7)
    for ny, W in ((200, 10.0), (128, 6.0), (64, 14.0)):
        rv, rl = 0.01 + 0.1 * rng.random(), 5 + 3 * rng.random()
        prof = SW.planar_profile(ny, rv, rl, W) * (1 + 1e-3 * rng.standard_normal(ny))
        assert SW.interface_width(prof, rv, rl) == OL.interface_width(prof, rv, rl)
        psi = np.sqrt(prof) * (1 + 0.1 * rng.random())
        assert SW.surface_tension(psi) == pytest.approx(OL.surface_tension_planar(psi), rel=1e-13)
        assert SW.density_error(rv * 1.05, rv) == pytest.approx(OL.vapor_density_error(rv * 1.05, rv), rel=1e-14)
