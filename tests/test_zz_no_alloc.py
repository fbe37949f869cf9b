"""The allocation-free EDT entry point (relo_edt_noalloc) through the C ABI.

It exists for callers that may not allocate device memory once running (a
real-time loop that allocates only at start-up, or a framework that owns all
device memory through its own pool); its scratch is a fixed file-scope device
array.  Its output must equal the EDT table of the regular entry point
(relo_load_map + relo_map_tables_dev) and the oracle's exact EDT, call after
call, since the scratch is reused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def relo():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_01219_gb300 as relo
    return relo


def grids():
    import workloads
    rng = np.random.default_rng(42)
    for shape in ((1, 1), (65, 1), (1, 77)):      # one segment, one column, one row
        yield np.where(rng.random(shape) < 0.3, 100, 0).astype(np.int8)
    yield np.zeros((40, 37), np.int8)            # no occupied cell: every d2 is -1
    yield workloads.make_room(3, n=64)
    g = np.where(rng.random((333, 517)) < 0.01, 100, 0).astype(np.int8)
    g[rng.random(g.shape) < 0.02] = -1
    yield g
    yield workloads.make_office(7, n=1024)


def regular_d2(relo, g):
    ctx = relo.Relo()
    mid = ctx.load_map(g, 0.05)
    d2, _, _ = ctx.map_tables(mid, g.shape)
    out = d2.cpu().numpy()
    ctx.close()
    return out


def noalloc_d2(relo, g, null_stream=False):
    import torch
    L = relo.lib()
    gd = torch.tensor(g, device="cuda")
    out = torch.full(g.shape, -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    if null_stream:
        stream = None                               # NULL: the default stream
    else:
        s = torch.cuda.current_stream().cuda_stream
        stream = ctypes.c_void_p(s if s else 1)     # 1: the legacy default stream handle
    rc = L.relo_edt_noalloc(ctypes.c_void_p(gd.data_ptr()), g.shape[1], g.shape[0], ctypes.c_void_p(out.data_ptr()),
                            stream)
    assert rc == relo.OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_edt_matches_regular_entry_point_two_calls_in_a_row(relo):
    import oracle
    for g in grids():
        want = regular_d2(relo, g)
        first = noalloc_d2(relo, g)
        second = noalloc_d2(relo, g)
        assert np.array_equal(first, want)
        assert np.array_equal(second, want)
        exact = oracle.edt(g)
        assert np.array_equal(first.astype(np.int64), exact)
        if not (g >= 65).any():
            assert (first == -1).all()


def test_noalloc_edt_on_the_null_stream(relo):
    import workloads
    g = workloads.make_room(4, n=96)
    got = noalloc_d2(relo, g, null_stream=True)
    assert np.array_equal(got, regular_d2(relo, g))


def test_noalloc_edt_rejects_oversized_maps(relo):
    import torch
    L = relo.lib()
    gd = torch.zeros((8, 1025), dtype=torch.int8, device="cuda")
    out = torch.empty((8, 1025), dtype=torch.int32, device="cuda")
    rc = L.relo_edt_noalloc(ctypes.c_void_p(gd.data_ptr()), 1025, 8, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == relo.E_INVALID_ARG
    tall = torch.zeros((1025, 8), dtype=torch.int8, device="cuda")
    out2 = torch.empty((1025, 8), dtype=torch.int32, device="cuda")
    rc = L.relo_edt_noalloc(ctypes.c_void_p(tall.data_ptr()), 8, 1025, ctypes.c_void_p(out2.data_ptr()), None)
    assert rc == relo.E_INVALID_ARG
    rc = L.relo_edt_noalloc(None, 8, 8, ctypes.c_void_p(out2.data_ptr()), None)
    assert rc == relo.E_INVALID_ARG
