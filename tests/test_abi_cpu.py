"""CPU checks of the C ABI: the library builds, loads, exports every entry point declared in include/dg.h,
and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dg\w*)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    from paper_2112_10517_gb300 import build
    return build.build()


def test_library_exports_every_declared_entry_point(built):
    lib = ctypes.CDLL(built["libdg.so"])
    names = declared_functions("dg.h")
    assert "dg_init" in names and "dg_rhs" in names and "dg_step" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_peaks_library_exports(built):
    lib = ctypes.CDLL(built["libdgpeaks.so"])
    for n in declared_functions("dg_peaks.h"):
        assert hasattr(lib, n), n


def test_argument_errors_without_gpu(built):
    from paper_2112_10517_gb300 import dg
    assert dg.dg_status_string(dg.DG_ERR_ARG) == b"invalid argument"
    ctx = ctypes.c_void_p()
    mesh = dg.DgMesh()
    opts = dg.DgOpts()
    opts.gamma = 1.4
    mesh.ndims = 4  # invalid
    assert dg.dg_init(ctypes.byref(ctx), ctypes.byref(mesh), 3, None, ctypes.byref(opts)) == dg.DG_ERR_ARG
    mesh.ndims = 3
    for i in range(3):
        mesh.nelem[i] = 2
        mesh.lo[i] = -1.0
        mesh.hi[i] = 1.0
    assert dg.dg_init(ctypes.byref(ctx), ctypes.byref(mesh), 9, None, ctypes.byref(opts)) == dg.DG_ERR_UNSUPPORTED
    assert dg.dg_init(ctypes.byref(ctx), ctypes.byref(mesh), 0, None, ctypes.byref(opts)) == dg.DG_ERR_UNSUPPORTED
    opts.gamma = 1.0
    assert dg.dg_init(ctypes.byref(ctx), ctypes.byref(mesh), 3, None, ctypes.byref(opts)) == dg.DG_ERR_ARG
    opts.gamma = 1.4
    opts.launch = 2
    assert dg.dg_init(ctypes.byref(ctx), ctypes.byref(mesh), 3, None, ctypes.byref(opts)) == dg.DG_ERR_ARG
    opts.launch = -1
    assert dg.dg_init(ctypes.byref(ctx), ctypes.byref(mesh), 3, None, ctypes.byref(opts)) == dg.DG_ERR_ARG
    opts.launch = dg.DG_LAUNCH_SERIAL
    opts.staging = 3
    assert dg.dg_init(ctypes.byref(ctx), ctypes.byref(mesh), 3, None, ctypes.byref(opts)) == dg.DG_ERR_ARG
    opts.staging = dg.DG_STAGING_DIRECT
    # log-mean options: out of range, or combinations without a kernel, are rejected before any device call
    init = lambda: dg.dg_init(ctypes.byref(ctx), ctypes.byref(mesh), 3, None, ctypes.byref(opts))
    opts.precompute_logs = 2
    assert init() == dg.DG_ERR_ARG
    opts.precompute_logs = 0
    opts.logmean = 3
    assert init() == dg.DG_ERR_ARG
    opts.logmean, opts.precompute_logs = dg.DG_LOGMEAN_ALG, 1  # precomputed logs need the default log mean
    assert init() == dg.DG_ERR_UNSUPPORTED
    opts.logmean, opts.volume_flux = 0, dg.DG_VOL_SHIMA  # the Shima flux has no logarithmic means
    assert init() == dg.DG_ERR_UNSUPPORTED
    opts.precompute_logs, opts.volume_flux = 0, dg.DG_VOL_RANOCHA
    opts.volume_flux = 2
    assert init() == dg.DG_ERR_ARG
    opts.volume_flux = dg.DG_VOL_RANOCHA
    mesh.hi[1] = -2.0  # empty box
    assert dg.dg_init(ctypes.byref(ctx), ctypes.byref(mesh), 3, None, ctypes.byref(opts)) == dg.DG_ERR_ARG
    mesh.hi[1] = 1.0
    mesh.nelem[2] = 0  # no elements
    assert dg.dg_init(ctypes.byref(ctx), ctypes.byref(mesh), 3, None, ctypes.byref(opts)) == dg.DG_ERR_ARG
    assert dg.dg_rhs(None, None, None, 0.0, None) == dg.DG_ERR_ARG
    assert dg.dg_step(None, None, None, 0.0, 0.1, 0, None) == dg.DG_ERR_ARG
    assert dg.dg_check_status(None) == dg.DG_ERR_ARG
    assert dg.dg_launch_count(None) == -1
    dg.dg_free(None)  # no-op


def test_noalloc_rejects_misaligned_arrays_before_any_device_call(built):
    """dg_rhs_noalloc reads u, invJ and the metric terms and writes du and the flag in whole elements: a pointer
    that is not a multiple of its element size is refused before the library touches a device (the fake
    addresses below are never dereferenced)."""
    from paper_2112_10517_gb300 import dg
    nelem = (ctypes.c_int * 3)(2, 2, 2)
    state = 2 * 2 * 2 * 5 * 64 * 8  # bytes of one state array: 8 elements, 5 variables, 64 nodes
    u, du, invJ = 0x100000, 0x100000 + 2 * state, 0x100000 + 4 * state
    ja64, ja32, flag = 0x100000 + 6 * state, 0x100000 + 6 * state + 4, 0x100000 + 8 * state

    def call(precision, ja, fl, uu=u):
        return dg.dg_rhs_noalloc(3, nelem, 3, precision, dg.DG_SURF_EC_LLF, 1.4, ctypes.c_void_p(uu),
                                 ctypes.c_void_p(ja), ctypes.c_void_p(invJ), ctypes.c_void_p(du),
                                 ctypes.c_void_p(fl), None)

    assert call(dg.DG_FP64, ja32, flag) == dg.DG_ERR_ARG      # FP64 metric terms 4 bytes off an 8-byte boundary
    assert call(dg.DG_FP32, ja32 + 2, flag) == dg.DG_ERR_ARG  # FP32 metric terms 2 bytes off
    assert call(dg.DG_FP64, ja64, flag + 2) == dg.DG_ERR_ARG  # the int flag 2 bytes off
    assert call(dg.DG_FP64, ja64, flag, uu=u + 4) == dg.DG_ERR_ARG  # the state 4 bytes off


def test_mesh_size_limits_are_rejected_before_any_device_call(built):
    # the kernels index nodes with 32-bit offsets: E * (p+1)^nd * (nd+2) must stay below 2^31 (DG_ERR_UNSUPPORTED),
    # and every direction holds at most 2^20 elements (DG_ERR_ARG); both checks come before any device call
    from paper_2112_10517_gb300 import dg
    ctx = ctypes.c_void_p()
    opts = dg.DgOpts()
    opts.gamma = 1.4

    def init(nelem, p, part=None):
        mesh = dg.DgMesh()
        mesh.ndims = len(nelem)
        for i, n in enumerate(nelem):
            mesh.nelem[i], mesh.lo[i], mesh.hi[i] = n, -1.0, 1.0
        if part is None:
            return dg.dg_init(ctypes.byref(ctx), ctypes.byref(mesh), p, None, ctypes.byref(opts))
        pa = dg.DgPart()
        pa.begin, pa.end = part
        return dg.dg_init_part(ctypes.byref(ctx), ctypes.byref(mesh), p, ctypes.byref(opts), ctypes.byref(pa))

    assert 189 ** 3 * 64 * 5 > 2 ** 31 - 1 > 188 ** 3 * 64 * 5
    assert init([189, 189, 189], 3) == dg.DG_ERR_UNSUPPORTED
    assert 128 ** 3 * 512 * 5 > 2 ** 31 - 1
    assert init([128, 128, 128], 7) == dg.DG_ERR_UNSUPPORTED
    assert init([1 << 21, 1], 1) == dg.DG_ERR_ARG                # more than 2^20 elements along x
    # a slab counts its own layers plus the ghost layer: 2 own layers of 1536 x 1536 elements at p = 3 would fit,
    # with the ghost layer they do not
    layer = 1536 * 1536 * 64 * 5
    assert 2 * layer <= 2 ** 31 - 1 < 3 * layer
    assert init([1536, 1536, 4], 3, part=(0, 2)) == dg.DG_ERR_UNSUPPORTED
    assert not ctx.value
