"""rsi_set_allocator: with a caller allocator set, every device allocation
of the library goes through it (handle storage, the segment-order and
inside-test workspaces, host-path staging, the adjoint's accumulator) and is
freed through it; results do not change; a failing or misaligned allocator
gives an error instead of a fault."""
import numpy as np
import pytest
import torch

import paper_2209_02878_gb300 as rsi
from paper_2209_02878_gb300 import RSIError, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


class Counting:
    """Torch's caching allocator with a ledger of live pointers."""

    def __init__(self, offset=0, fail=False):
        self.live, self.n_alloc, self.n_free = {}, 0, 0
        self.offset, self.fail = offset, fail

    def alloc(self, nbytes, device, stream):
        if self.fail:
            return 0
        p = torch.cuda.caching_allocator_alloc(nbytes + self.offset, device=device, stream=stream)
        self.live[p + self.offset] = p
        self.n_alloc += 1
        return p + self.offset

    def free(self, p, device, stream):
        torch.cuda.caching_allocator_delete(self.live.pop(p))
        self.n_free += 1


@pytest.fixture
def counting():
    c = Counting()
    rsi.set_allocator(c.alloc, c.free)
    yield c
    rsi.set_allocator(None, None)


def test_every_allocation_goes_through_the_callbacks(counting):
    mesh, seg = synth.workload_small_bool()
    V, T, A, B = dev(mesh.V), dev(mesh.T), dev(seg.A), dev(seg.B)
    rsi.set_allocator(None, None)
    ref = rsi.BVH(V, T).intersect(A, B, "nearest")
    ref_sorted = rsi.BVH(V, T).intersect(A, B, "count")["count"].cpu()
    rsi.set_allocator(counting.alloc, counting.free)
    bvh = rsi.BVH(V, T)
    assert counting.n_alloc == 1                      # the handle's storage
    got = bvh.intersect(A, B, "nearest")
    cnt = bvh.intersect(A, B, "count", launch=dict(sort_bits=16))["count"]   # order workspace
    host = bvh.intersect_host(A.cpu(), B.cpu(), "bool")                     # staging
    inside = bvh.points_inside(A)                                           # inside workspace
    gV = torch.zeros_like(V)
    rsi.intersect_backward(V, T, A, B, got["tri"], grad_point=torch.ones_like(A), grad_V=gV)
    torch.cuda.synchronize()
    assert counting.n_alloc >= 5
    assert counting.n_free >= 1                       # the adjoint's accumulator
    np.testing.assert_array_equal(got["tri"].cpu(), ref["tri"].cpu())
    np.testing.assert_array_equal(cnt.cpu(), ref_sorted)
    np.testing.assert_array_equal(host["flag"].numpy(), (ref_sorted > 0).numpy().astype(np.uint8))
    assert inside.shape[0] == A.shape[0]
    # handles keep their allocator: switching back does not change where
    # their memory is returned
    rsi.set_allocator(None, None)
    bvh.close()
    torch.cuda.synchronize()
    assert counting.live == {} and counting.n_alloc == counting.n_free


def test_failing_allocator_gives_out_of_memory():
    c = Counting(fail=True)
    rsi.set_allocator(c.alloc, c.free)
    try:
        mesh, _ = synth.workload_small_bool()
        with pytest.raises(RSIError) as ei:
            rsi.BVH(dev(mesh.V), dev(mesh.T))
        assert ei.value.code == 3  # RSI_ERR_OOM
    finally:
        rsi.set_allocator(None, None)


def test_misaligned_allocator_is_refused():
    c = Counting(offset=16)
    rsi.set_allocator(c.alloc, c.free)
    try:
        mesh, _ = synth.workload_small_bool()
        with pytest.raises(RSIError):
            rsi.BVH(dev(mesh.V), dev(mesh.T))
        torch.cuda.synchronize()
        assert c.live == {} and c.n_alloc == c.n_free == 1   # handed back
    finally:
        rsi.set_allocator(None, None)


def test_torch_allocator_round_trip():
    mesh, seg = synth.workload_small_bool()
    V, T, A, B = dev(mesh.V), dev(mesh.T), dev(seg.A), dev(seg.B)
    ref = rsi.BVH(V, T).intersect(A, B, "count")["count"].cpu()
    rsi.use_torch_allocator()
    try:
        before = torch.cuda.memory_allocated()
        bvh = rsi.BVH(V, T)
        assert torch.cuda.memory_allocated() > before     # the handle lives in torch's pool
        np.testing.assert_array_equal(bvh.intersect(A, B, "count")["count"].cpu(), ref)
        bvh.close()
    finally:
        rsi.use_torch_allocator(False)
