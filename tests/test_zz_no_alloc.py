"""pald_cohesion_noalloc, the pass-2 entry point for callers that must not
allocate device memory (for example because their own pool already owns the
device memory, or because an allocation's implicit synchronisation is not
acceptable in their loop).  It keeps its scratch in a fixed array built into
the library, so it is limited to n <= 2048.

It runs the same kernels as pald_cohesion, so its output must be the same
bits.  The test also watches the device's memory while it runs: the stream-
ordered pool's high-water mark (which pald_cohesion's own scratch does
raise), the free device memory and torch's allocator must not move.

The file name makes pytest collect it last.  It must pass on its own in a
fresh process and after every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2307_16652_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu

PALD_ERR_NOT_SYMMETRIC = 2
POOL_USED_CURRENT, POOL_USED_HIGH = 0x7, 0x8  # cudaMemPoolAttr values


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    binding.lib()


class PoolWatch:
    """The default stream-ordered memory pool of the current device, read
    through the CUDA runtime the library itself is linked against."""

    def __init__(self):
        self.rt = ctypes.CDLL("libcudart.so.13")
        self.pool = ctypes.c_void_p()
        dev = torch.cuda.current_device()
        assert self.rt.cudaDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.rt.cudaMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)  # resets the high-water mark to the current use
        assert self.rt.cudaMemPoolSetAttribute(self.pool, POOL_USED_HIGH, ctypes.byref(zero)) == 0

    def snapshot(self):
        torch.cuda.synchronize()
        free, _ = torch.cuda.mem_get_info()
        return {"pool_high": self.get(POOL_USED_HIGH), "pool_used": self.get(POOL_USED_CURRENT),
                "free": free, "torch": torch.cuda.memory_allocated()}


def _case(n, kind):
    D_np = inputs.plain_matrix(n) if kind == "plain" else inputs.tie_heavy_matrix(n, hi=9)
    D = torch.from_numpy(D_np).cuda()
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    binding.pald_focus(D, U)
    ref = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_cohesion(D, U, ref)
    return D, U, ref


@pytest.mark.parametrize("n,kind", [(2048, "plain"), (701, "tie")])
def test_noalloc_matches_pald_cohesion_on_two_calls(n, kind):
    D, U, ref = _case(n, kind)
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    watch = PoolWatch()
    binding.pald_cohesion_noalloc(D, U, C)  # first call on the device: looks up the array's address
    torch.cuda.synchronize()
    watch.reset_high()
    before = watch.snapshot()
    for _ in range(2):  # the fixed scratch keeps the previous call's contents
        C.fill_(-1.0)
        torch.cuda.synchronize()
        watch.reset_high()
        binding.pald_cohesion_noalloc(D, U, C)
        after = watch.snapshot()
        assert after == before, f"device memory moved during the call: {before} -> {after}"
        assert torch.equal(C, ref), "not the bits pald_cohesion gives"


def test_the_memory_watch_sees_an_allocating_call():
    # control: pald_cohesion takes its scratch from the stream-ordered pool,
    # which raises the pool's high-water mark that the test above watches
    D, U, _ = _case(512, "plain")
    C = torch.empty((512, 512), dtype=torch.float32, device="cuda")
    watch = PoolWatch()
    torch.cuda.synchronize()
    watch.reset_high()
    before = watch.get(POOL_USED_HIGH)
    binding.pald_cohesion(D, U, C)
    torch.cuda.synchronize()
    assert watch.get(POOL_USED_HIGH) >= before + 512 * 512 * 4


def test_noalloc_validation_then_a_valid_call():
    # validation writes its summary into the shared array and reads it back
    n = 300
    D, U, ref = _case(n, "plain")
    bad = D.clone()
    bad[3, 7] = bad[3, 7] * 2.0  # no longer symmetric
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.PaldError) as err:
        binding.pald_cohesion_noalloc(bad, U, C, validate=True)
    assert err.value.status == PALD_ERR_NOT_SYMMETRIC
    binding.pald_cohesion_noalloc(D, U, C, validate=True)
    torch.cuda.synchronize()
    assert torch.equal(C, ref)


def test_noalloc_rejects_orders_beyond_its_array():
    o = binding.PaldOpts(0, 0, -1, 0)
    fake = ctypes.c_void_p(256)  # never touched: the size check comes first
    st = binding.lib().pald_cohesion_noalloc(fake, fake, 2049, fake, ctypes.byref(o), None)
    assert st == 8  # PALD_ERR_UNSUPPORTED
    assert "unsupported" in binding.pald_status_string(st)
