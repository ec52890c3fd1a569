"""xamg_hier_save / xamg_hier_load: the frozen hierarchy as a byte blob.

CPU (host-only hierarchies): the blob round-trips byte for byte, the loaded
hierarchy exports the same levels as the saved one, and malformed blobs
(wrong magic, every truncation, trailing bytes, corrupted lengths and
indices) are rejected with XAMG_ERR_INVALID_ARG.  GPU: a loaded hierarchy
solves bit for bit like the one it was saved from.
"""
import struct

import numpy as np
import pytest

from paper_2103_07329_gb300 import binding as B
from paper_2103_07329_gb300 import problems as P


def host_hier(A, **kw):
    return B.Hierarchy(A, device_upload=0, **kw)


@pytest.mark.parametrize("name,N", [("p7", 12), ("p27", 7), ("p7", 3)])
def test_roundtrip_is_exact(name, N):
    A = P.poisson7(N) if name == "p7" else P.poisson27(N)
    h = host_hier(A)
    blob = h.save()
    g = B.Hierarchy.load(blob)
    assert not g.on_device
    assert g.levels == h.levels and g.n == h.n
    assert g.save() == blob  # every field survives
    for l in range(h.levels):
        a, b = h.level_export(l), g.level_export(l)
        assert a["n"] == b["n"]
        for k in ("A", "P"):
            if a[k] is None:
                assert b[k] is None
            else:
                assert all(np.array_equal(x, y) for x, y in zip(a[k], b[k]))
        for k in ("cf", "cheb"):
            assert (a[k] is None and b[k] is None) or np.array_equal(a[k], b[k])
    lu_a, piv_a = h.coarse_export()
    lu_b, piv_b = g.coarse_export()
    assert np.array_equal(lu_a, lu_b) and np.array_equal(piv_a, piv_b)


def test_size_query_and_short_buffer():
    import ctypes as C
    h = host_hier(P.poisson7(6))
    L = B.lib()
    n = C.c_size_t()
    assert L.xamg_hier_save(h.handle, None, 0, C.byref(n)) == 0 and n.value > 0
    buf = C.create_string_buffer(n.value)
    m = C.c_size_t()
    assert L.xamg_hier_save(h.handle, buf, n.value - 1, C.byref(m)) == B.ERR_INVALID_ARG
    assert m.value == n.value


def load_code(blob: bytes) -> int:
    import ctypes as C
    L = B.lib()
    out = C.c_void_p()
    buf = C.create_string_buffer(blob, max(len(blob), 1))
    rc = L.xamg_hier_load(buf, len(blob), C.byref(out))
    if rc == 0:
        L.xamg_destroy(out)
    return rc


def test_malformed_blobs_are_rejected():
    blob = host_hier(P.poisson7(8)).save()
    assert load_code(blob) == 0
    # wrong magic, version, byte order
    for pos in (0, 8, 12):
        bad = bytearray(blob)
        bad[pos] ^= 0xFF
        assert load_code(bytes(bad)) == B.ERR_INVALID_ARG
    # every truncation and one trailing byte
    cuts = sorted(set(list(range(0, 80)) + list(np.linspace(80, len(blob) - 1, 60).astype(int))))
    for c in cuts:
        assert load_code(blob[:c]) == B.ERR_INVALID_ARG, c
    assert load_code(blob + b"\0") == B.ERR_INVALID_ARG
    # level count 0 and huge
    head = 8 + 4 + 4 + 8 + 4 * 4 + 8 + 8 + 4 * 3  # magic, version, order, parameters
    for L in (0, 1 << 30):
        bad = bytearray(blob)
        bad[head:head + 4] = struct.pack("<I", L)
        assert load_code(bytes(bad)) == B.ERR_INVALID_ARG
    # the first level's rowptr length field inflated past the blob
    off = head + 4 + 4 + 4 + 4 + 4  # L, cheb_steps, nc, A.n, A.ncols
    bad = bytearray(blob)
    bad[off:off + 8] = struct.pack("<Q", 1 << 40)
    assert load_code(bytes(bad)) == B.ERR_INVALID_ARG
    # a column index out of range in the first level's A
    n0 = struct.unpack_from("<i", blob, head + 12)[0]
    col_off = off + 8 + 4 * (n0 + 1) + 8  # rowptr (length, data), col length
    bad = bytearray(blob)
    bad[col_off:col_off + 4] = struct.pack("<i", n0)
    assert load_code(bytes(bad)) == B.ERR_INVALID_ARG


@pytest.mark.gpu
def test_loaded_hierarchy_solves_bitwise():
    torch = pytest.importorskip("torch")
    from paper_2103_07329_gb300 import build as build_mod
    build_mod.build()
    A = P.poisson7(24)
    h = B.Hierarchy(A)
    g = B.Hierarchy.load(h.save())
    assert g.on_device
    Bm = torch.from_numpy(P.rhs_uniform(A.n, 5, 3)).cuda()
    for prec in (B.PREC_FP64, B.PREC_FP32):
        X1 = torch.empty_like(Bm)
        X2 = torch.empty_like(Bm)
        s1 = h.solve(Bm, X1, precond=prec)
        s2 = g.solve(Bm, X2, precond=prec)
        assert torch.equal(X1, X2) and np.array_equal(s1.iters, s2.iters)
        assert s1.rc == 0


def test_device_blob_without_a_device_fails_cleanly():
    # a host-only blob with its upload flag set: where no GPU is present the
    # load returns XAMG_ERR_CUDA (no crash, nothing leaked); with a GPU it
    # uploads like any other load
    import ctypes as C
    blob = bytearray(host_hier(P.poisson7(6)).save())
    flag = 8 + 4 + 4 + 8 + 4 * 4 + 8 + 8 + 4 + 4  # magic, version, order, parameters before device_upload
    assert struct.unpack_from("<i", blob, flag)[0] == 0
    blob[flag:flag + 4] = struct.pack("<i", 1)
    L = B.lib()
    out = C.c_void_p()
    buf = C.create_string_buffer(bytes(blob), len(blob))
    rc = L.xamg_hier_load(buf, len(blob), C.byref(out))
    has_gpu = False
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        pass
    if has_gpu:
        assert rc == 0
        L.xamg_destroy(out)
    else:
        assert rc == B.ERR_CUDA and not out.value


def test_random_corruptions_never_crash():
    # seeded single-byte corruptions and random-length prefixes anywhere in the
    # blob: every load either succeeds (a value changed but the structure
    # still checks out), returns XAMG_ERR_INVALID_ARG, or -- when the byte
    # set the upload flag and no GPU is present -- XAMG_ERR_CUDA
    blob = host_hier(P.poisson7(7)).save()
    ok = (0, B.ERR_INVALID_ARG, B.ERR_CUDA)
    rng = np.random.default_rng(2024)
    for _ in range(300):
        bad = bytearray(blob)
        pos = int(rng.integers(0, len(blob)))
        bad[pos] = int(rng.integers(0, 256))
        assert load_code(bytes(bad)) in ok, pos
    for _ in range(100):
        cut = int(rng.integers(0, len(blob)))
        tail = bytes(rng.integers(0, 256, size=int(rng.integers(0, 64)), dtype=np.uint8))
        assert load_code(blob[:cut] + tail) in ok, cut
