"""Host-side checks of the C ABI (no GPU needed): exports, argument
validation, status strings, byte accounting and allocation fault injection."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lfp.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__._cuda_build_module().build()
    from paper_2507_14624_gb300 import lfp
    return lfp


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lfp_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_entry_point_is_exported(lib):
    names = declared_functions()
    assert {"lfp_create_grid", "lfp_upload_probes", "lfp_render", "lfp_render_backward"} <= set(names)
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lfp_\w+)", out))
    assert set(names) <= exported


def _desc(lfp, **kw):
    d = lfp.lfp_grid_desc()
    d.nx = d.ny = d.nz = 2
    d.spacing, d.N, d.M = 1.0, 64, 16
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("field,value", [("nx", 1), ("N", 63), ("M", 3), ("M", 128), ("N", 48 * 0 + 100),
                                         ("spacing", 0.0), ("spacing", float("nan")), ("radiance_fmt", 7),
                                         ("max_steps", -1), ("eye_eps", -1.0), ("eye_lookup", 2),
                                         ("traversal", 2), ("traversal", -1)])
def test_invalid_descriptors_are_rejected(lib, field, value):
    d = _desc(lib, **{field: value})
    if field == "N" and value == 100:
        d.M = 16  # 100 % 16 != 0
    h = ctypes.c_void_p(123)
    st = lib.raw_call("lfp_create_grid", ctypes.byref(d), ctypes.byref(h))
    assert st == lib.LFP_ERR_INVALID_ARG
    assert h.value is None  # *out is cleared on failure
    b = ctypes.c_ulonglong()
    assert lib.raw_call("lfp_grid_bytes", ctypes.byref(d), ctypes.byref(b)) == lib.LFP_ERR_INVALID_ARG


@pytest.mark.parametrize("dims,ok", [((1, 1, 1), True), ((2, 1, 1), True), ((2, 2, 1), True), ((2, 2, 2), True),
                                     ((3, 3, 1), False), ((0, 1, 1), False)])
def test_nearest_traversal_takes_one_to_eight_probes(lib, dims, ok):
    """Sec. 4.3's mode for fewer than 8 probes: any 1..8 probes (no cells
    needed); the grid traversal keeps nx, ny, nz >= 2."""
    d = _desc(lib, nx=dims[0], ny=dims[1], nz=dims[2], traversal=lib.LFP_TRAVERSAL_NEAREST)
    b = ctypes.c_ulonglong()
    want = lib.LFP_OK if ok else lib.LFP_ERR_INVALID_ARG
    assert lib.raw_call("lfp_grid_bytes", ctypes.byref(d), ctypes.byref(b)) == want
    d.traversal = lib.LFP_TRAVERSAL_GRID
    want = lib.LFP_OK if min(dims) >= 2 else lib.LFP_ERR_INVALID_ARG
    assert lib.raw_call("lfp_grid_bytes", ctypes.byref(d), ctypes.byref(b)) == want


def test_null_arguments_are_rejected(lib):
    L = lib
    assert L.raw_call("lfp_create_grid", None, None) == L.LFP_ERR_INVALID_ARG
    assert L.raw_call("lfp_upload_probes", None, 0, 1, None, None) == L.LFP_ERR_INVALID_ARG
    assert L.raw_call("lfp_render", None, None, 1, None, None, None, None, None) == L.LFP_ERR_INVALID_ARG
    assert L.raw_call("lfp_render_backward", None, None, 1, None, None, None, None, None, None) == L.LFP_ERR_INVALID_ARG
    assert L.raw_call("lfp_set_radiance", None, None, None) == L.LFP_ERR_INVALID_ARG
    assert L.raw_call("lfp_check_flags", None, None) == L.LFP_ERR_INVALID_ARG
    assert L.raw_call("lfp_render_to_host_async", None, None, 1, None, None, None) == L.LFP_ERR_INVALID_ARG
    assert L.raw_call("lfp_sync_host", None) == L.LFP_ERR_INVALID_ARG
    assert L.raw_call("lfp_build_probes_from_points", None, 0, 1, None, 0.0, None) == L.LFP_ERR_INVALID_ARG
    assert L.raw_call("lfp_read_probes", None, 0, 1, None, None, None, None) == L.LFP_ERR_INVALID_ARG
    assert L.raw_call("lfp_pick_levels", None, 1, None, 1, None) == L.LFP_ERR_INVALID_ARG
    assert L.raw_call("lfp_render_levels", None, 1, None, 1, None, None, None) == L.LFP_ERR_INVALID_ARG
    assert L.raw_call("lfp_render_backward_levels", None, 1, None, 1, None, None, None, None, None, 0,
                      None) == L.LFP_ERR_INVALID_ARG
    L.lfp_destroy_grid(None)  # NULL-safe


def test_status_strings(lib):
    for s in (0, 1, 2, 3, 4, 5, 6, 100):
        assert len(lib.lfp_status_string(s)) >= 2
    assert lib.lfp_status_string(999) == "unknown status"


def test_grid_bytes_accounting(lib):
    """Storage per probe: N^2 (4 distance + normal + radiance) bytes, 8
    bytes (min, max) per block of every skip level (N = 256 with blocks of
    4, 8, 16 and 32 texels has 64^2 + 32^2 + 16^2 + 8^2 blocks) and 16 bytes
    for the least distance of each map quadrant. FP16 texels halve the
    normal (8 -> 4) and radiance (16 -> 8) bytes."""
    d = _desc(lib, nx=4, ny=4, nz=4, N=256, M=16)
    blocks = 64 * 64 + 32 * 32 + 16 * 16 + 8 * 8
    assert lib.lfp_grid_bytes(d) == 64 * (256 * 256 * (4 + 8 + 16) + blocks * 8 + 16)
    d.radiance_fmt = d.normal_fmt = lib.LFP_TEXEL_F16
    assert lib.lfp_grid_bytes(d) == 64 * (256 * 256 * (4 + 4 + 8) + blocks * 8 + 16)


@pytest.mark.parametrize("N,M,want", [
    (256, 16, [4, 8, 16, 32]),   # k = 16: k/4, k/2, k, 2k
    (512, 32, [4, 8, 16, 32]),
    (64, 16, [2, 4, 8]),         # k/4 = 1 is no skip
    (48, 16, [3, 6]),            # k = 3: k/4, k/2 not whole
    (192, 16, [3, 6, 12, 24]),
    (6, 2, [3]),                 # 2k = 6 leaves one block per side (odd)
    (256, 256, [1, 2]),          # the descriptor's own k = 1 is kept
    (96, 2, [12, 24, 48]),       # 2k = 96 leaves one block per side
    (40, 4, [5, 10, 20]),        # k = 10: k/4 not whole, k/2 = 5, 2k = 20 (two blocks per side)
])
def test_skip_levels_of_a_descriptor(lib, N, M, want):
    """The skip levels: block sides k/4, k/2, 2k (k = N/M) that are whole,
    >= 2, divide N into an even number of blocks, plus k itself."""
    got = lib.lfp_skip_blocks(_desc(lib, N=N, M=M))
    assert got == want
    assert N // M in got
    for k in got:
        assert N % k == 0 and ((N // k) % 2 == 0 or k == N // M)


def test_skip_levels_reject_invalid_arguments(lib):
    b = (ctypes.c_int * lib.LFP_MAX_SKIP_LEVELS)()
    n = ctypes.c_int()
    assert lib.raw_call("lfp_skip_blocks", ctypes.byref(_desc(lib, M=3)), b, ctypes.byref(n)) == lib.LFP_ERR_INVALID_ARG
    assert lib.raw_call("lfp_skip_blocks", None, b, ctypes.byref(n)) == lib.LFP_ERR_INVALID_ARG
    assert lib.raw_call("lfp_skip_blocks", ctypes.byref(_desc(lib)), None, ctypes.byref(n)) == lib.LFP_ERR_INVALID_ARG


def test_allocation_fault_injection_returns_oom_without_a_device(lib):
    """LFP_FAULT_ALLOC_FAIL=1 fails the first device allocation inside
    lfp_create_grid before any CUDA call: the status is OOM and the handle
    stays NULL (run in a fresh process so the allocation counter starts at 0)."""
    code = (
        "import ctypes, sys; sys.path.insert(0, %r)\n"
        "from paper_2507_14624_gb300 import lfp\n"
        "d = lfp.lfp_grid_desc(); d.nx = d.ny = d.nz = 2; d.spacing = 1.0; d.N = 64; d.M = 16\n"
        "h = ctypes.c_void_p(7)\n"
        "st = lfp.raw_call('lfp_create_grid', ctypes.byref(d), ctypes.byref(h))\n"
        "print(st, h.value)\n" % ROOT)
    env = dict(os.environ, LFP_FAULT_ALLOC_FAIL="1", CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=120)
    assert out.returncode == 0, out.stderr
    st, h = out.stdout.split()
    assert int(st) == 2 and h == "None"


def test_checked_library_exports_the_same_entry_points(lib):
    """liblfp_checked.so (every texel index tested) is a drop-in for
    liblfp.so: it exports every entry point the header declares."""
    import __graft_entry__
    path = __graft_entry__._cuda_build_module().build(checked=True)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lfp_\w+)", out))
    assert set(declared_functions()) <= exported
