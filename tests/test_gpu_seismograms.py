"""The seismogram chain of Sec. 4.1.2 through the C ABI (lsm_seismograms) against the oracle's chain.

Both sides: for f_k = k df the background field of the source, the LS solve, the three components
at the receiver nodes, and the Ricker-weighted inverse Fourier sum.  The FP64 chain is solved to
relres 1e-12 on both sides (traces within 1e-9 of the largest sample); the mixed-precision chain to
1e-8 (within 1e-6).  Waves of 7 frequencies leave a ragged last wave.
"""
import numpy as np
import pytest

import synthetic as sy
from oracle import synthesis as osyn
from paper_2301_12836_gb300 import lsm

from gpu_helpers import handle, host

pytestmark = pytest.mark.gpu

NF, DF, NT, DT, FP, T0 = 24, 2.0, 250, 2e-3, 12.0, 0.08
XS = np.array([75.0, 75.0, 75.0])
REC = [(ix, iy, 1) for ix in (2, 7, 13) for iy in (3, 8, 12)]


@pytest.fixture(scope="module")
def oracle_chain():
    med = sy.inclusion_medium(16, 10.0)
    tr, U, its = osyn.seismograms(med, NF, DF, sy.explosion(), XS, REC, NT, DT, FP, T0, tol=1e-12)
    return med, tr, its


@pytest.mark.parametrize("precision,tol,bound", [(lsm.LSM_FP64, 1e-12, 1e-9), (lsm.LSM_MIXED, 1e-8, 1e-6)])
def test_seismograms_match_the_oracle_chain(oracle_chain, precision, tol, bound):
    med, want, its_o = oracle_chain
    h = handle(med, 2 * np.pi * DF, precision=precision, tol=tol)
    code, tr, its, rr = lsm.lsm_seismograms(h, NF, DF, sy.explosion(), XS, REC, NT, DT, FP, T0, wave=7)
    assert code == lsm.LSM_OK
    assert its[0] == 0 and all(i > 0 for i in its[1:]) and max(rr) <= tol
    if precision == lsm.LSM_FP64:
        assert all(abs(a - b) <= 1 for a, b in zip(its[1:], its_o[1:]))
    got = host(tr)
    assert got.shape == want.shape == (len(REC), 3, NT)
    assert np.abs(got - want).max() <= bound * np.abs(want).max()


def test_seismograms_reject_a_receiver_outside_the_grid():
    med = sy.inclusion_medium(16, 10.0)
    h = handle(med, 2 * np.pi * DF)
    with pytest.raises(lsm.LSMError) as e:
        lsm.lsm_seismograms(h, 4, DF, sy.explosion(), XS, [(0, 0, 16)], 10, DT, FP, T0)
    assert e.value.code == lsm.LSM_ERR_ARG
