"""A caller's device allocator (dem_params.alloc / free; here blocks of
PyTorch's caching allocator allocated on the context's stream, so that a block
given back is reused only after the work queued on that stream) serves every
buffer of a context: a deterministic run on it is bit-identical to the same
run on the library's own stream-ordered allocator, and every block it handed
out is given back when the context closes.  A block that is not 256-byte
aligned (the kernels move 16- and 32-byte records) fails the call before any
kernel sees it, and is given back."""
import numpy as np
import pytest

import paper_2307_03445_gb300 as dem
from paper_2307_03445_gb300 import scenes
from paper_2307_03445_gb300.capi import DemError

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class TorchBlocks:
    """Device blocks from PyTorch, shifted by `shift` bytes from the start of
    their storage (PyTorch's own blocks are 512-byte aligned)."""

    def __init__(self, stream, shift=0):
        self.stream, self.shift, self.live, self.handed = stream, shift, {}, 0

    def alloc(self, n):
        with torch.cuda.stream(self.stream):
            t = torch.empty(n + 512, dtype=torch.uint8, device="cuda")
        p = t.data_ptr() + self.shift
        self.live[p] = t
        self.handed += 1
        return p

    def free(self, p):
        del self.live[p]


def _run(scene, stream, allocator=None):
    sim = dem.Simulation(scene, margin=1e-4, rebuild_interval=5, stream=stream,
                         allocator=allocator)
    sim.set_deterministic(True)
    sim.step(12)
    state = sim.state()
    a, b, u, ws, ww, uw = sim.contacts()
    sim.close()
    return list(state) + [a, b, u, ws, ww, uw]


@pytest.mark.parametrize("prec", [scenes.PREC_FP64, scenes.PREC_FP32])
def test_caller_allocator_run_equals_the_library_allocator(prec):
    scene = scenes.packed_scene(5, 300, precision=prec)
    s = torch.cuda.Stream()
    ref = _run(scene, s.cuda_stream)
    blocks = TorchBlocks(s)
    got = _run(scene, s.cuda_stream, (blocks.alloc, blocks.free))
    torch.cuda.synchronize()
    assert blocks.handed > 0
    assert not blocks.live, "blocks not given back when the context closed"
    for r, g in zip(ref, got):
        np.testing.assert_array_equal(r, g)


def test_misaligned_block_fails_the_call_and_is_given_back():
    scene = scenes.packed_scene(5, 50, precision=scenes.PREC_FP32)
    s = torch.cuda.Stream()
    blocks = TorchBlocks(s, shift=16)
    with pytest.raises(DemError) as err:
        dem.Simulation(scene, margin=1e-4, stream=s.cuda_stream, allocator=(blocks.alloc, blocks.free))
    assert err.value.code == -2  # DEM_ERR_OOM
    assert blocks.handed > 0 and not blocks.live
