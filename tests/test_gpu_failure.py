"""Failure detection without a GPU fault: the grid barrier of the persistent
master solve is a bounded wait.  A cooperative launch in which one block never
arrives must end with the other block giving up after the poll limit, the
barrier marked broken, DAO_ETIMEOUT reported, and the device usable for the
next plan."""
import ctypes as C
import time

import pytest

import phantom as P
from _helpers import need_cuda

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(120)]


@pytest.fixture(scope="module")
def torch():
    t = need_cuda()
    from paper_1003_5402_gb300 import build
    build.build()
    return t


def test_barrier_wait_gives_up_and_device_stays_usable(torch):
    from paper_1003_5402_gb300 import Plan, binding
    lib = binding.load()
    gave_up, passed = C.c_int32(-1), C.c_int32(-1)
    t0 = time.perf_counter()
    st = lib.dao_check_bounded_wait(0, C.byref(gave_up), C.byref(passed))
    waited = time.perf_counter() - t0
    assert st == binding.DAO_ETIMEOUT, lib.dao_last_error().decode()
    assert gave_up.value == 1 and passed.value == 0
    assert waited < 60.0
    case = P.make_case(P.spec_micro())
    with Plan(case, stream=torch.cuda.current_stream().cuda_stream) as plan:
        st, n, trace = plan.solve(4)
        assert n == 4 and all(trace[k + 1] <= trace[k] for k in range(3))
