"""The allocation-free keys + sort entry point (nbody_sort_keys_noalloc) against the context
path (nbody_build_tree + nbody_get_keys), called through the C ABI.

That entry point serves callers that cannot call cudaMalloc (runtimes with a fixed
device-memory budget, real-time loops that must not block in the allocator); its scratch is one
file-scope device array shared by every call, so this test makes two calls in a row on different
inputs and checks that the second is not affected by what the first left in the array, at the
largest size it accepts and at the smallest ones.  This file is collected last."""
import ctypes

import numpy as np
import pytest

import ics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2203_08966_gb300 as nb  # noqa: E402

MAX_N = 262144


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    return nb.load_library()


def _noalloc(lib, pos, mass):
    n = mass.shape[0]
    tp = torch.from_numpy(pos).cuda()
    tm = torch.from_numpy(mass).cuda()
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    st = lib.nbody_sort_keys_noalloc(ctypes.c_void_p(tp.data_ptr()), ctypes.c_void_p(tm.data_ptr()),
                                     n, ctypes.c_void_p(keys.data_ptr()),
                                     ctypes.c_void_p(ids.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return keys.cpu().numpy().view(np.uint64), ids.cpu().numpy().view(np.uint32)


def _context(pos, mass):
    n = mass.shape[0]
    with nb.Context(n) as ctx:
        ctx.build_tree(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda())
        return ctx.keys(n)


def test_noalloc_matches_context_path_on_two_calls(lib):
    first = ics.two_plummer(MAX_N, seeds=(14, 15))
    second = ics.plummer(77777, 16)
    k1, i1 = _noalloc(lib, first[0], first[2])
    k2, i2 = _noalloc(lib, second[0], second[2])
    r1 = _context(first[0], first[2])
    r2 = _context(second[0], second[2])
    assert np.array_equal(k1, r1[0]) and np.array_equal(i1, r1[1])
    assert np.array_equal(k2, r2[0]) and np.array_equal(i2, r2[1])


@pytest.mark.parametrize("n", [1, 2, 3, 4096, 4097])
def test_noalloc_small_and_tile_edge_sizes(lib, n):
    pos, _, mass = ics.plummer(n, 20 + n % 7)
    k, i = _noalloc(lib, pos, mass)
    r = _context(pos, mass)
    assert np.array_equal(k, r[0]) and np.array_equal(i, r[1])


def test_noalloc_rejects_sizes_beyond_its_maximum(lib):
    n = MAX_N + 1
    buf = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert lib.nbody_sort_keys_noalloc(p, p, n, p, p, None) == 1
    assert lib.nbody_sort_keys_noalloc(p, p, -1, p, p, None) == 1
    assert lib.nbody_sort_keys_noalloc(None, p, 10, p, p, None) == 1
