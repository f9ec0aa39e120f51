"""Failure detection without a GPU fault: the bounded waits of the tensor-core
kernels give up after a device-time limit, set the state's asynchronous
error word, and the next synchronising call reports QSIM_E_TIMEOUT; the
context and the state stay usable. The wait is made to run out on an
mbarrier that nothing arrives at (qsim_selftest_wait_timeout), never by
faulting or hanging the GPU."""
import time

import numpy as np
import pytest

import oracle
from paper_2304_14969_gb300 import workloads as W

pytestmark = pytest.mark.gpu

QSIM_E_TIMEOUT = 4


@pytest.fixture(scope="module")
def Q():
    from paper_2304_14969_gb300 import qsim
    qsim.lib()
    return qsim


def test_wait_timeout_is_reported_and_state_stays_usable(Q):
    n = 12
    x = W.gaussian_state(n, 3)
    g = W.random_1q_circuit(n, 40, 3)
    st = Q.State(n, 1)
    st.upload(x)
    t0 = time.perf_counter()
    Q.qsim_selftest_wait_timeout(st.h, 50_000_000)          # 50 ms of device time
    with pytest.raises(Q.QsimError) as e:
        Q.qsim_synchronize(st.h)
    assert e.value.status == QSIM_E_TIMEOUT
    assert time.perf_counter() - t0 >= 0.04                   # the wait did run for its limit
    Q.qsim_synchronize(st.h)                                  # reported once, then cleared
    # the state and the context still work: amplitudes untouched, gates run
    assert np.max(np.abs(st.download() - x)) == 0.0
    st.run(Q.Circuit(n, g), mode=0, relabel=1)
    y = st.download()
    ref = oracle.apply_circuit(x, g)
    assert 1 - abs(np.vdot(ref, y)) ** 2 <= 1e-12
    st.close()


def test_wait_timeout_reported_by_a_reduction(Q):
    st = Q.State(8, 0)
    Q.qsim_selftest_wait_timeout(st.h, 1_000_000)
    with pytest.raises(Q.QsimError) as e:
        st.norm()
    assert e.value.status == QSIM_E_TIMEOUT
    assert abs(st.norm() - 1.0) < 1e-6
    st.close()


def test_wait_timeout_limit_checked_on_host(Q):
    st = Q.State(4, 0)
    for bad in (0, 999, 10_000_000_001):
        with pytest.raises(Q.QsimError) as e:
            Q.qsim_selftest_wait_timeout(st.h, bad)
        assert e.value.status == 1
    st.close()
