import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def ob():
    """The oracle module, compiled once per session."""
    from oracle import bop
    bop.build()
    return bop


def oracle_model(p):
    from oracle import bop
    return bop.Model(p.norb, tuple(p.b0), p.r0, p.lam, p.rc, p.dc, p.onsite0, p.rep_A, p.rep_p, p.onsite_s)


def oracle_settings(r):
    from oracle import bop
    return bop.Settings(n_e=r.n_e, n_mom=r.n_mom, n_exp=r.n_exp, n_spin=r.n_spin, scf=r.scf,
                        eta=r.eta, scf_tol=r.scf_tol, scf_max_it=r.scf_max_it,
                        stoner_I=r.stoner_I, m_mix=r.m_mix, m0=r.m0, dos_floor=r.dos_floor,
                        mixer=r.mixer, mix_history=r.mix_history, scf_response=r.scf_response,
                        bandwidth=None if r.bandwidth == "gershgorin" else
                        bop.Bandwidth(r.bandwidth, r.bw_beta, r.bw_a, r.bw_b), J_ii=r.J_ii,
                        r_path=r.r_path, noncollinear=r.noncollinear)
