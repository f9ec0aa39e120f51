"""The allocation-free inner product, for callers that cannot let the
library allocate device memory (their device memory belongs to another
allocator, or their loop must not wait in the driver's allocator).

It must agree with qsim_inner_product, which keeps its partial sums in
library-allocated scratch, on two calls in a row (the shared fixed scratch
keeps the previous call's contents), and with the FP64 oracle's inner
product of the same kets. Sizes include n = 24, where the sum kernel's grid
is capped at the array's 1024 partial rows and every thread loops several
times. Once the entry point has run on a device, further calls leave the
device's free memory unchanged: they allocate nothing. This file is
collected last on purpose, and passes alone in a fresh process as well."""
import ctypes as C

import numpy as np
import pytest

import oracle
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
@pytest.mark.parametrize("n", [1, 7, 20, 24])
def test_noalloc_matches_inner_product_twice(Q, dt, n):
    a = Q.State(n, dt)
    b = Q.State(n, dt)
    npdt = np.complex64 if dt == 0 else np.complex128
    for call in range(2):
        xa = W.gaussian_state(n, 10 * call + 1).astype(npdt)
        xb = W.gaussian_state(n, 10 * call + 2).astype(npdt)
        a.upload(xa)
        b.upload(xb)
        ref = a.inner(b)
        orc = oracle.inner(xa.astype(np.complex128), xb.astype(np.complex128))
        out = (C.c_double * 2)()
        Q.qsim_inner_product_noalloc(dev_ptr(Q, a), dev_ptr(Q, b), n, dt, None, out)
        got = complex(out[0], out[1])
        assert abs(got - ref) <= TOL[dt] * max(1.0, abs(ref)), (call, got, ref)
        assert abs(got - orc) <= TOL[dt] * max(1.0, abs(orc)), (call, got, orc)
    a.close()
    b.close()


def test_noalloc_leaves_free_memory_unchanged(Q):
    """After a first call on the device (which may load the library's kernels),
    calls change neither the device's free memory nor torch's pool."""
    import torch
    n = 22
    a = Q.State(n, 0)
    b = Q.State(n, 0)
    a.upload(W.gaussian_state(n, 3))
    b.upload(W.gaussian_state(n, 4))
    out = (C.c_double * 2)()
    Q.qsim_inner_product_noalloc(dev_ptr(Q, a), dev_ptr(Q, b), n, 0, None, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    vals = []
    for _ in range(3):
        Q.qsim_inner_product_noalloc(dev_ptr(Q, a), dev_ptr(Q, b), n, 0, None, out)
        vals.append(complex(out[0], out[1]))
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert torch.cuda.memory_reserved() == reserved0
    assert vals[0] == vals[1] == vals[2]
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
