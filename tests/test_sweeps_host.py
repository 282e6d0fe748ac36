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


def test_kappa_for_surface_tension_inverts_the_one_minus_kappa_law():
    """Sec. V's recipe: kappa such that (1 - kappa) gamma_0 = gamma_target; a lower
    surface tension needs a negative kappa, a higher one a positive kappa below 1."""
    for g0, gt in ((4.86e-3, 6.32e-3), (6.3e-3, 3.1e-3), (1.0, 1.0)):
        k = SW.kappa_for_surface_tension(gt, g0)
        assert (1 - k) * g0 == pytest.approx(gt, rel=1e-14)
        assert k < 1
    assert SW.kappa_for_surface_tension(6.32e-3, 4.86e-3) < 0
    for bad in ((0.0, 1.0), (1.0, 0.0), (-1.0, 1.0)):
        with pytest.raises(ValueError):
            SW.kappa_for_surface_tension(*bad)
