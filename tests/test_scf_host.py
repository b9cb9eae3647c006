"""Host-only entry point of the self-consistent closure: fe_occupations (Fermi-Dirac
filling by bisection) against the oracle, and its argument checks.  Needs no GPU."""
import numpy as np
import pytest

from oracle import scf


@pytest.fixture(scope="module")
def fe():
    import paper_2504_00998_gb300 as fe
    fe.load()
    return fe


@pytest.mark.parametrize("kT,ne", [(1e-3, 23.0), (0.01, 40.0), (0.1, 7.5), (0.05, 0.0)])
def test_occupations_match_oracle(fe, kT, ne):
    from paper_2504_00998_gb300 import scf as fscf
    eps = np.sort(np.random.default_rng(5).uniform(-2.0, 1.0, 40))
    occ, mu = fscf.occupations(eps, ne, kT)
    occ_r, mu_r = scf.occupations(eps, ne, kT)
    np.testing.assert_allclose(occ, occ_r, rtol=0, atol=1e-12)
    assert abs(occ.sum() - ne) <= 1e-10
    if ne > 0:
        assert abs(mu - mu_r) <= 1e-10


def test_occupations_reject_bad_arguments(fe):
    from paper_2504_00998_gb300 import scf as fscf
    with pytest.raises(fe.FeError):
        fscf.occupations(np.zeros(4), 9.0, 0.01)      # more than 2 n electrons
    with pytest.raises(fe.FeError):
        fscf.occupations(np.zeros(4), 2.0, 0.0)       # kT must be positive
