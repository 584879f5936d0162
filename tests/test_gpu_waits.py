"""Failure detection of the bounded device waits, without a GPU fault.

The grid barrier of the batched sweep and the mbarrier waits of the
tensor-core kernels give up after a bounded number of polls, set an error flag
the host reads and return, so a lost arrival ends in an error status instead
of a hung GPU.  The self-test entry point makes each wait run out on an event
that never comes (a block that leaves without arriving, an mbarrier nobody
arrives at) with a short poll limit, beside a control where the event comes.
After it the device must still take work: a sweep on a fresh context still
matches the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_26361_gb300 import ebit
from paper_2509_26361_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_waits_give_up_and_report_it():
    code, rep = ebit.ebit_selftest_bounded_waits()
    # barrier met (result, flag), barrier with a block absent (result, flag),
    # mbarrier with and without the arrival
    assert rep == [1, 0, 0, 1, 1, 0], rep
    assert code == ebit.EBIT_OK
    torch.cuda.synchronize()


def test_device_keeps_working_after_a_wait_gave_up():
    code, _ = ebit.ebit_selftest_bounded_waits()
    assert code == ebit.EBIT_OK
    n = 16
    w = W.fourier_spheres(n=n, seed=11, count=2, rmin=0.15, rmax=0.25, steps=1)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    g = ebit.Grid(n, n, n)
    g.init(dev(w.phi), dev(w.phi_faces))
    g.sweep(0, dev(w.u[0]), 0.5 * g.h)
    cb, _ = g.get_state()
    o, _ = oracle.sweep(oracle.init(w.phi, w.phi_faces), 0, w.u[0], 0.5)
    assert np.array_equal(cb.cpu().numpy(), o.cb)
    g.close()
