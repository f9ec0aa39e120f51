"""The allocation-free inner product, for callers that cannot let the
library allocate device memory (their device memory belongs to another
allocator, or their loop must not wait in the driver's allocator).

It must agree with qsim_inner_product, which keeps its partial sums in
library-allocated scratch, on two calls in a row (the shared fixed scratch
keeps the previous call's contents). This file is collected last on
purpose, and passes alone in a fresh process as well."""
import ctypes as C

import numpy as np
import pytest

from paper_2304_14969_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 2e-6, 1: 1e-13}


@pytest.fixture(scope="module")
def Q():
    from paper_2304_14969_gb300 import build, qsim
    build.build()
    qsim.lib()
    return qsim


def dev_ptr(Q, st):
    p = C.c_void_p()
    Q.qsim_device_ptr(st.h, C.byref(p))
    return p


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [1, 7, 20])
def test_noalloc_matches_inner_product_twice(Q, dt, n):
    a = Q.State(n, dt)
    b = Q.State(n, dt)
    for call in range(2):
        a.upload(W.gaussian_state(n, 10 * call + 1))
        b.upload(W.gaussian_state(n, 10 * call + 2))
        ref = a.inner(b)
        out = (C.c_double * 2)()
        Q.qsim_inner_product_noalloc(dev_ptr(Q, a), dev_ptr(Q, b), n, dt, None, out)
        got = complex(out[0], out[1])
        assert abs(got - ref) <= TOL[dt] * max(1.0, abs(ref)), (call, got, ref)
    a.close()
    b.close()


def test_noalloc_rejects_bad_sizes(Q):
    a = Q.State(3, 0)
    out = (C.c_double * 2)()
    for n in (0, 37):
        with pytest.raises(Q.QsimError) as e:
            Q.qsim_inner_product_noalloc(dev_ptr(Q, a), dev_ptr(Q, a), n, 0, None, out)
        assert e.value.status == 1
    a.close()
