"""The energy sweep's measurement through the C ABI against the oracle: the full-step energies of a
short toy-scenario run (s = 3, nu = 0.5) follow Algorithm 2 of the oracle, so RVITE (Eq. 4) agrees."""
import numpy as np
import pytest

import oracle
from oracle import respa

pytestmark = pytest.mark.gpu


def test_toy_rvite_matches_the_oracle(gpu_lib):
    from paper_2507_11172_gb300 import sweeps
    x, L, v = sweeps.toy_state()
    nu, s, iters, dt = 0.5, 3, 60, 0.001
    r_gpu, e_gpu, _ = sweeps.run_point(x, L, v, nu, s, iters, dt=dt, equil=0, precision=gpu_lib.MD_FP64)
    st = respa.State(x.copy(), v.copy(), L)
    f2b, f3b = respa.lj_atm_forces(L, 1.0, 1.0, 2.5, nu, 2.5)
    e_ref = []
    for _ in range(iters // s):
        respa.run(st, 1, s, s * dt, f2b, f3b)
        e_ref.append((oracle.kinetic(st.v), st.u2, st.u3))
    e_ref = np.asarray(e_ref)
    scale = np.abs(e_ref).sum(1)
    assert np.all(np.abs(e_gpu.sum(1) - e_ref.sum(1)) <= 1e-10 * scale)
    assert abs(r_gpu - respa.rvite(e_ref.sum(1), e_ref[:, 0])) <= 1e-6 * respa.rvite(e_ref.sum(1), e_ref[:, 0])
