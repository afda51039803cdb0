"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/rtlbfs.h, and its host-only entry points agree with the
oracle; argument errors come back as status codes, and the binding checks the
buffers the library writes into."""
import ctypes as C

import numpy as np
import pytest

from paper_2202_13449_gb300 import capi


def test_library_exports_every_declared_function():
    L = capi.lib()
    declared = capi.header_functions()
    assert len(declared) >= 19
    missing = [f for f in declared if not hasattr(L, f)]
    assert missing == []


@pytest.mark.parametrize("n,L,phi", [(512, 512.0, 2.0), (64, 64.0, 0.0), (80, 1.0, 1.8),
                                     (33, 7.5, 2.5)])
def test_tanh_faces_matches_oracle(orc, n, L, phi):
    np.testing.assert_array_equal(capi.tanh_faces(n, L, phi), orc.tanh_faces(n, L, phi))


def test_host_argument_errors_are_status_codes():
    L = capi.lib()
    out = np.empty(4)
    assert L.rtlbfs_tanh_faces(0, 1.0, 1.0, out.ctypes.data_as(C.POINTER(C.c_double))) == capi.ERR_ARG
    assert L.rtlbfs_tanh_faces(3, -1.0, 1.0, out.ctypes.data_as(C.POINTER(C.c_double))) == capi.ERR_ARG
    # a null handle is rejected, never dereferenced
    assert L.rtlbfs_step(None, 1) == capi.ERR_ARG
    assert L.rtlbfs_set_params(None, 1e3, 0.71, 0.1, 0.5) == capi.ERR_ARG
    assert L.rtlbfs_last_error(None) == b"null handle"
    L.rtlbfs_destroy(None)
    h = C.c_void_p()
    xf = np.arange(5.0)
    bad = np.array([0.0, 1.0, 1.0, 2.0, 3.0])
    dp = C.POINTER(C.c_double)
    assert L.rtlbfs_create_mesh(4, 4, xf.ctypes.data_as(dp), bad.ctypes.data_as(dp), 0,
                                C.byref(h)) != capi.OK
    assert not h.value


def test_op_counts_of_the_step():
    """The ALU work measure: the face arithmetic of the kernels counted on
    the host (data-independent, so fixed), two faces plus the per-cell
    terms per cell-update."""
    face, cell, sfu = capi.op_counts()
    assert face == int(face) and 150 <= face <= 200
    assert cell == 2 * face + 95
    assert sfu == 2 * 1 + 4  # one reciprocal per face; rho^{n+1}, two roots, one reciprocal


def test_op_counts_of_the_tlbfs_stage():
    face_r, cell_r, _ = capi.op_counts(capi.RTLBFS)
    face_t, cell_t, sfu_t = capi.op_counts(capi.TLBFS)
    assert cell_t == 2 * face_t + 95 and sfu_t == 6
    assert face_t > 1.5 * face_r  # nine equilibria and their moments per face
    with pytest.raises(capi.RTLBFSError):
        capi.op_counts(2)


def test_raw_output_buffers_are_checked_before_the_library_writes():
    """The state-record readers write through a bare pointer: the binding
    refuses a buffer that is too small, strided or read-only."""
    ok = np.zeros(64, dtype=np.uint8)
    assert capi._raw_out(ok, 64) is not None
    assert capi._raw_out(np.zeros(8), 64).nbytes == 64  # any dtype, counted in bytes
    assert capi._raw_out(bytearray(80), 64).nbytes == 80
    ro = np.zeros(64, dtype=np.uint8)
    ro.flags.writeable = False
    for bad in (np.zeros(63, dtype=np.uint8), np.zeros((8, 16), dtype=np.uint8)[:, ::2], ro):
        with pytest.raises(ValueError):
            capi._raw_out(bad, 64)
