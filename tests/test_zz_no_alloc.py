"""pod_sample_noalloc (the allocation-free column draw for callers that
cannot allocate device memory) against pod_sample, through the C ABI.

Runs last (file name) so that a first-failure run has already run every
other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import isma as O  # noqa: E402
from paper_1905_05107_gb300 import build, pod  # noqa: E402

build.build()
DEV = torch.device("cuda:0")


def _draw(fn, w, mask, c, seed, t):
    idx = torch.full((c,), -1, dtype=torch.int32, device=DEV)
    g = torch.zeros(1, dtype=torch.int32, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    st = fn(ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(mask.data_ptr()), w.shape[0], c, seed, t, 0,
            ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(g.data_ptr()), stream)
    assert st == pod.POD_OK, pod.strerror(st)
    torch.cuda.synchronize()
    return idx[: int(g.item())].cpu().numpy(), mask.cpu().numpy().copy()


@pytest.mark.parametrize("n,c", [(2000, 40), (65536, 300), (37, 4096)])
def test_noalloc_sampler_matches_allocating_entry_point_twice(n, c):
    L = pod.lib()
    rng = np.random.default_rng(n + c)
    vals = rng.random(n) ** 2
    vals[rng.random(n) < 0.05] = 0.0
    mask0 = rng.random(n) < 0.9
    mask0[0] = True
    w = torch.from_numpy(O.quantize(vals, mask0).view(np.int64)).to(DEV)
    m_ref = torch.from_numpy(mask0.astype(np.uint8)).to(DEV)
    m_new = m_ref.clone()
    for call, (seed, t) in enumerate([(0x5107 + n, 3), (0xBEEF + c, 4)]):
        ref_idx, ref_mask = _draw(L.pod_sample, w, m_ref, c, seed, t)
        new_idx, new_mask = _draw(L.pod_sample_noalloc, w, m_new, c, seed, t)
        assert np.array_equal(new_idx, ref_idx), "call %d" % call
        assert np.array_equal(new_mask, ref_mask), "call %d" % call


def test_noalloc_sampler_leaves_device_memory_unchanged():
    """After the first call on the device (which looks up, and under lazy
    module loading places, the fixed arrays), further calls change neither
    the device's free memory nor what the caching allocator holds."""
    L = pod.lib()
    n, c = 4000, 64
    w = torch.ones(n, dtype=torch.int64, device=DEV)
    mask = torch.ones(n, dtype=torch.uint8, device=DEV)
    idx = torch.zeros(c, dtype=torch.int32, device=DEV)
    g = torch.zeros(1, dtype=torch.int32, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)

    def call(t):
        st = L.pod_sample_noalloc(ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(mask.data_ptr()), n, c, 1, t, 0,
                                  ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(g.data_ptr()), stream)
        assert st == pod.POD_OK, pod.strerror(st)

    call(0)                                  # set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(DEV)
    held0 = torch.cuda.memory_reserved(DEV)
    for t in range(1, 4):
        mask.fill_(1)
        call(t)
    torch.cuda.synchronize()
    assert int(g.item()) > 0
    free1, _ = torch.cuda.mem_get_info(DEV)
    assert free1 == free0 and torch.cuda.memory_reserved(DEV) == held0


def test_noalloc_sampler_rejects_sizes_beyond_its_arrays():
    L = pod.lib()
    n = (1 << 16) + 1
    w = torch.ones(n, dtype=torch.int64, device=DEV)
    mask = torch.ones(n, dtype=torch.uint8, device=DEV)
    idx = torch.zeros(8, dtype=torch.int32, device=DEV)
    g = torch.zeros(1, dtype=torch.int32, device=DEV)
    st = L.pod_sample_noalloc(ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(mask.data_ptr()), n, 8, 1, 0, 0,
                              ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(g.data_ptr()), None)
    assert st == pod.POD_EUNSUPPORTED
