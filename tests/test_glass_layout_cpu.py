"""The library's glass layout (host code behind steps_glass_layout: Eq. 16-18)
against the oracle's, and its argument checks.  No GPU needed."""
import math

import numpy as np
import pytest

from oracle import glass as og
from paper_1811_05903_gb300 import steps

RHO = 3.0 / (8.0 * math.pi)


@pytest.mark.parametrize("scheme,D,R,nr,ns,rc", [(0, 60.0, 342.45, 30, 64, 45.0), (1, 100.0, 342.45, 40, 96, 0.0),
                                                 (0, 10.0, 1000.0, 7, 5, 3.0), (1, 5.0, 20.0, 1, 3, 0.0)])
def test_layout_matches_oracle(scheme, D, R, nr, ns, rc):
    steps.load(build_if_missing=True)
    n, ni, mi, edges, masses = steps.steps_glass_layout(steps.glass_spec(scheme, D, R, nr, ns, rc, RHO))
    e_ref, m_ref, ni_ref, mi_ref = og.layout(scheme, D, R, nr, ns, rc, RHO)
    assert ni == ni_ref and n == ni_ref + nr * ns
    np.testing.assert_allclose(edges, e_ref, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(masses, m_ref, rtol=1e-12)
    assert mi == pytest.approx(mi_ref, rel=1e-12)


@pytest.mark.parametrize("kw", [dict(D_s=0.0), dict(R_sim=-1.0), dict(n_radial=0), dict(n_shell=0),
                                dict(r_c=0.0), dict(r_c=400.0), dict(scheme=2), dict(rho_bar=math.nan)])
def test_layout_rejects_bad_specs(kw):
    steps.load(build_if_missing=True)
    args = dict(scheme=0, D_s=60.0, R_sim=342.45, n_radial=30, n_shell=64, r_c=45.0, rho_bar=RHO)
    args.update(kw)
    with pytest.raises(steps.StepsError) as e:
        steps.steps_glass_layout(steps.glass_spec(**args))
    assert e.value.status == steps.STEPS_EINVAL
