"""The allocation-free P2G entry point, checked against a context's P2G.

tsim_p2g_noalloc serves callers that cannot allocate device memory (a
plug-in whose host application owns all device memory, a real-time loop that
must not touch the allocator, a fixed memory budget): it works in a fixed
scratch array the library reserves on every GPU.  This test calls it through
the C ABI twice in a row, on two different particle states, and compares
each result with the grid that a context computes for the same state
(tsim_write_particles + tsim_read_grid) within the tolerances of the other
parity tests.  Its file name makes pytest collect it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2405_02914_gb300 import inputs as I
from paper_2405_02914_gb300 import tsim as T

pytestmark = pytest.mark.gpu


def _state(sc, seed):
    rng = np.random.default_rng(seed)
    x, tag = I.gel_particles(sc.gel)
    n = x.shape[0]
    v = (0.02 * rng.standard_normal((n, 3))).astype(np.float32)
    Cm = (5.0 * rng.standard_normal((n, 9))).astype(np.float32)
    F = (np.eye(3).reshape(9) + 0.02 * rng.standard_normal((n, 9))).astype(np.float32)
    return x, v, Cm, F, tag


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_p2g_matches_context_on_two_calls():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    L = T.load()
    stream = torch.cuda.current_stream()
    for call, (dims, seed) in enumerate([((13, 9, 5), 21), ((16, 12, 6), 22)]):
        sc = I.scene_small(cx=dims[0], cy=dims[1], cz=dims[2], seed=seed)
        state = _state(sc, seed)
        sim = T.Sim(sc, states=[state])
        ref = sim.grid()
        sim.close()
        dev = [torch.from_numpy(a).cuda() for a in state[:4]]
        nn = int(np.prod(sc.gel.nodes))
        out = torch.full((nn, 4), float("nan"), device="cuda")   # must be overwritten
        gel, mat = T.gel_desc(sc.gel), T.material_desc(sc.mat)
        rc = L.tsim_p2g_noalloc(C.byref(gel), C.byref(mat), C.c_float(sc.solver.dt),
                                C.c_void_p(dev[0].data_ptr()), C.c_void_p(dev[1].data_ptr()),
                                C.c_void_p(dev[2].data_ptr()), C.c_void_p(dev[3].data_ptr()),
                                state[0].shape[0], C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == 0, L.tsim_last_error().decode()
        g = out.cpu().numpy()
        assert np.isfinite(g).all(), call
        assert _rel_l2(g[:, 0], ref[:, 0]) < 1e-6, call
        assert _rel_l2(g[:, 1:], ref[:, 1:]) < 1e-4, call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    L = T.load()
    sc = I.scene_small(cx=4, cy=4, cz=2)
    gel, mat = T.gel_desc(sc.gel), T.material_desc(sc.mat)
    buf = torch.zeros(16, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    rc = L.tsim_p2g_noalloc(C.byref(gel), C.byref(mat), C.c_float(1e-5), p, p, p, p, (1 << 20) + 1, p, None)
    assert rc == 1 and b"1048576" in L.tsim_last_error()
    big = T.gel_desc(I.Gel(256, 256, 64, 1e-3))                # more cell blocks than the scratch holds
    rc = L.tsim_p2g_noalloc(C.byref(big), C.byref(mat), C.c_float(1e-5), p, p, p, p, 8, p, None)
    assert rc == 1 and b"cell blocks" in L.tsim_last_error()


def test_noalloc_rejects_misaligned_and_host_arrays():
    """Arrays the kernels cannot use are refused before any GPU work: a grid
    that is not 16-byte aligned (its float4 atomics would fault), a particle
    array off a 4-byte boundary, and host memory in place of device memory."""
    torch = pytest.importorskip("torch")
    L = T.load()
    sc = I.scene_small(cx=4, cy=4, cz=2)
    gel, mat = T.gel_desc(sc.gel), T.material_desc(sc.mat)
    n = sc.gel.n_particles
    nn = int(np.prod(sc.gel.nodes))
    # every buffer is large enough for the call, so nothing reads out of bounds
    parts = torch.zeros(n * 9 + 16, device="cuda")
    grid = torch.zeros(nn * 4 + 16, device="cuda")
    p = C.c_void_p(parts.data_ptr())
    dt = C.c_float(1e-5)

    def call(x, g):
        return L.tsim_p2g_noalloc(C.byref(gel), C.byref(mat), dt, x, p, p, p, n, g, None)

    rc = call(p, C.c_void_p(grid.data_ptr() + 4))
    assert rc == 1 and b"16-byte" in L.tsim_last_error()
    rc = call(C.c_void_p(parts.data_ptr() + 2), C.c_void_p(grid.data_ptr()))
    assert rc == 1 and b"4-byte" in L.tsim_last_error()
    host = np.zeros(nn * 4 + 16, dtype=np.float32)
    rc = call(p, C.c_void_p(host.ctypes.data))
    assert rc == 1 and b"device memory" in L.tsim_last_error()
    hx = np.zeros(n * 9 + 16, dtype=np.float32)
    rc = call(C.c_void_p(hx.ctypes.data), C.c_void_p(grid.data_ptr()))
    assert rc == 1 and b"device memory" in L.tsim_last_error()
    # the same aligned device buffers pass the checks (F = 0 then gives J = 0)
    assert call(p, C.c_void_p(grid.data_ptr())) == 4, L.tsim_last_error()
