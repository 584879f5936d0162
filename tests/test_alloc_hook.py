"""ebit_set_allocator: the library's device allocations through a caller's
allocator.  On the CPU: the argument check.  On the GPU: a context, a network
and a batch created through a counting allocator (torch's caching allocator
underneath) compute exactly what the default allocator gives, free every
pointer they took, and a refusal of any one allocation makes the creating
call return EBIT_ENOMEM with nothing left allocated.  The failures are made
on the host: the allocator returns NULL; no device fault is involved."""
import numpy as np
import pytest
import torch

from paper_2509_26361_gb300 import ebit
from paper_2509_26361_gb300 import workloads as W

N3 = (24, 16, 32)


class Counting:
    """alloc/free pair that records live pointers and refuses call `fail_at`."""

    def __init__(self, fail_at=0):
        self.calls = 0
        self.fail_at = fail_at
        self.live = {}

    def alloc(self, nbytes):
        self.calls += 1
        if self.calls == self.fail_at:
            return 0
        p = torch.cuda.caching_allocator_alloc(max(int(nbytes), 1))
        assert p % 256 == 0
        self.live[p] = nbytes
        return p

    def free(self, ptr):
        assert ptr in self.live, "freed a pointer this allocator did not return"
        del self.live[ptr]
        torch.cuda.caching_allocator_delete(ptr)


@pytest.fixture
def restore_default():
    yield
    ebit.ebit_set_allocator()


def test_exactly_one_null_function_is_rejected(restore_default):
    with pytest.raises(ebit.EbitError) as e:
        ebit.ebit_set_allocator(lambda n: 0, None)
    assert e.value.code == ebit.EBIT_EINVAL
    with pytest.raises(ebit.EbitError):
        ebit.ebit_set_allocator(None, lambda p: None)
    assert ebit.ebit_set_allocator() == ebit.EBIT_OK


def _problem():
    rng = np.random.default_rng(3)
    sp = [W.Sphere((0.3, 0.4, 0.5), 0.22), W.Sphere((0.7, 0.6, 0.35), 0.15)]
    phi, faces = W.sphere_phi_nodes_faces(N3, sp)
    u = W.fourier_velocity(N3, rng)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dev(phi), dev(faces), [dev(u[d]) for d in range(3)]


def _run(steps=2):
    phi, faces, u = _problem()
    g = ebit.Grid(*N3)
    g.init(phi, faces)
    for n in range(steps):
        g.step(n, u, 0.4 * g.h)
    cb, s = g.get_state()
    C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    g.front2vof(C, ebit.EBIT_FULL)
    g.sync()
    out = (cb.cpu(), s.cpu(), C.cpu(), g.counters())
    g.close()
    return out


@pytest.mark.gpu
def test_context_through_the_allocator_matches_the_default(restore_default):
    ref = _run()
    a = Counting()
    ebit.ebit_set_allocator(a.alloc, a.free)
    got = _run()
    assert a.calls > 30 and not a.live
    for x, y in zip(ref[:3], got[:3]):
        assert torch.equal(x, y)
    assert ref[3] == got[3]


@pytest.mark.gpu
def test_every_refused_context_allocation_is_rolled_back(restore_default):
    a = Counting()
    ebit.ebit_set_allocator(a.alloc, a.free)
    ebit.Grid(*N3).close()
    n = a.calls
    assert not a.live
    for k in range(1, n + 1):
        a = Counting(fail_at=k)
        ebit.ebit_set_allocator(a.alloc, a.free)
        with pytest.raises(ebit.EbitError) as e:
            ebit.Grid(*N3)
        assert e.value.code == ebit.EBIT_ENOMEM, k
        assert not a.live, f"allocation {k} refused: {len(a.live)} pointers leaked"
    ebit.ebit_set_allocator()
    ebit.Grid(*N3).close()


@pytest.mark.gpu
def test_refused_scratch_leaves_the_context_usable(restore_default):
    """get_state's scratch is the context's first allocation after creation:
    refusing it fails that call only; the next call allocates it and reads
    the same state as a default context."""
    ref = _run(steps=1)
    phi, faces, u = _problem()
    probe = Counting()
    ebit.ebit_set_allocator(probe.alloc, probe.free)
    ebit.Grid(*N3).close()
    a = Counting(fail_at=probe.calls + 1)
    ebit.ebit_set_allocator(a.alloc, a.free)
    g = ebit.Grid(*N3)
    ebit.ebit_set_allocator()  # the context keeps the counting pair
    g.init(phi, faces)
    g.step(0, u, 0.4 * g.h)
    with pytest.raises(ebit.EbitError) as e:
        g.get_state()
    assert e.value.code == ebit.EBIT_ENOMEM
    cb, s = g.get_state()
    assert torch.equal(cb.cpu(), ref[0]) and torch.equal(s.cpu(), ref[1])
    g.close()
    assert not a.live


@pytest.mark.gpu
def test_network_and_batch_allocations_are_rolled_back(restore_default):
    for make in (lambda: ebit.Mlp(), lambda: ebit.Batch([(16, 16, 16), (24, 16, 8)])):
        a = Counting()
        ebit.ebit_set_allocator(a.alloc, a.free)
        make().close()
        n = a.calls
        assert n >= 8 and not a.live
        for k in range(1, n + 1):
            a = Counting(fail_at=k)
            ebit.ebit_set_allocator(a.alloc, a.free)
            with pytest.raises(ebit.EbitError) as e:
                make()
            assert e.value.code == ebit.EBIT_ENOMEM, k
            assert not a.live, f"allocation {k} of {n} refused: {len(a.live)} pointers leaked"
