"""C-ABI contract checks that need no GPU: the library builds and loads, it
exports every entry point include/*.h declares, host-only planning agrees
with the oracle's independent segment schedule, and argument validation
rejects bad calls before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1705_10087_gb300 import build, capi

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load()


def declared_functions():
    text = "".join(open(os.path.join(INCLUDE, f)).read() for f in sorted(os.listdir(INCLUDE))
                   if f.endswith(".h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(csc_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_library_built_for_sm103a():
    out = os.popen(f"/usr/local/cuda/bin/cuobjdump --list-elf {build.LIB} 2>&1").read()
    assert "sm_103a" in out


@pytest.mark.parametrize("Tz,L,M", [(199_937, 64, 64), (199_937, 64, 256), (199_937, 64, 1024),
                                    (199_937, 64, 3072), (1985, 16, 10), (1985, 16, 1),
                                    (4_999_801, 200, 12_500), (7, 3, 7), (50, 1, 9)])
def test_plan_matches_oracle_schedule(lib, Tz, L, M):
    Mo, c, starts = capi.csc_plan(Tz, L, M)
    assert Mo == M
    assert c == oracle.phase_count(Tz, M, L)
    assert list(starts) == [oracle.segment_start(Tz, M, m) for m in range(M + 1)]


def test_plan_automatic_segments_use_two_phases(lib):
    for Tz, L in [(199_937, 64), (4_999_801, 200), (1985, 16)]:
        M, c, starts = capi.csc_plan(Tz, L, 0)
        assert np.diff(starts).min() >= 2 * L - 2
        assert c == 2


def test_plan_rejects_bad_sizes(lib):
    with pytest.raises(capi.CscError) as e:
        capi.csc_plan(10, 3, 11)
    assert e.value.status == capi.CSC_EINVAL
    assert "exceeds" in capi.csc_last_error_string()


def test_argument_validation_needs_no_device(lib):
    h = ctypes.c_void_p()
    D = np.zeros((2, 1, 4), np.float32)
    assert lib.csc_setup(ctypes.byref(h), D.ctypes.data, 0, 1, 4, None, None) == capi.CSC_EINVAL
    assert lib.csc_setup(ctypes.byref(h), D.ctypes.data, 2, 1, 513, None, None) == capi.CSC_EINVAL
    assert lib.csc_setup(ctypes.byref(h), None, 2, 1, 4, None, None) == capi.CSC_EINVAL
    for field, bad in (("launch_mode", 7), ("threads_per_segment", 64), ("init_mode", 4),
                       ("segment_width", -1)):
        o = capi.make_opts()
        setattr(o, field, bad)
        assert lib.csc_setup(ctypes.byref(h), D.ctypes.data, 2, 1, 4, ctypes.byref(o),
                             None) == capi.CSC_EINVAL, field
    assert lib.csc_init(None, D.ctypes.data, 10, 1.0, None) == capi.CSC_EINVAL
    assert lib.csc_kkt(None, D.ctypes.data, D.ctypes.data) == capi.CSC_EINVAL
    assert "csc_kkt" in capi.csc_last_error_string()
    assert lib.csc_solve(None, 1e-6, 10, None, None, None) == capi.CSC_EINVAL
    assert lib.csc_destroy(None) == capi.CSC_OK
    assert "csc_solve" in capi.csc_last_error_string()
    for polls in (0, -1, (1 << 22) + 1):
        assert lib.csc_check_wait_timeout(polls) == capi.CSC_EINVAL
    assert "polls" in capi.csc_last_error_string()


def test_default_opts(lib):
    o = capi.csc_opts()
    lib.csc_default_opts(ctypes.byref(o))
    assert (o.segments, o.updates_per_visit, o.max_resyncs) == (0, 0, -1)


@pytest.mark.parametrize("Tz,L,M", [(199_937, 64, 1024), (1985, 16, 10), (7, 3, 7), (50, 1, 9),
                                    (4_999_801, 200, 12_500), (1, 5, 1)])
def test_segment_of_closed_form(lib, Tz, L, M):
    # the kernels find a column's segment as floor(((t+1) M - 1) / Tz): the
    # inverse of the plan's starts floor(m Tz / M)
    _, _, starts = capi.csc_plan(Tz, L, M)
    t = np.unique(np.concatenate([np.arange(min(Tz, 3000)), starts[1:-1], starts[1:-1] - 1,
                                  np.array([Tz - 1])]))
    t = t[(t >= 0) & (t < Tz)]
    m = ((t + 1) * M - 1) // Tz
    assert np.all(starts[m] <= t) and np.all(t < starts[m + 1])


def test_binding_has_every_declared_function(lib):
    # the Python binding keeps the C names: one wrapper per declared entry point
    names = declared_functions()
    assert len(names) >= 30
    assert sorted(n for n in names if not callable(getattr(capi, n, None))) == []
    o = capi.csc_default_opts()
    assert (o.segments, o.updates_per_visit, o.max_resyncs) == (0, 0, -1)


def test_plain_c99_caller(lib, tmp_path):
    # include/*.h must be usable from C, not only C++: tests/c_abi_check.c is
    # compiled as C99 with warnings as errors, linked against libcsc.so and run
    # (host-only entry points and argument validation need no GPU)
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(build.LIB)
    exe = tmp_path / "c_abi_check"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I", os.path.join(root, "include"),
                           os.path.join(root, "tests", "c_abi_check.c"), "-L", libdir, "-lcsc",
                           "-Wl,-rpath," + libdir, "-o", str(exe)])
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0 and res.stdout.strip() == "ok", res.stdout + res.stderr
    # the binding's ctypes structures have the C layout: size and every offset
    res = subprocess.run([str(exe), "layout"], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stdout + res.stderr
    for line in res.stdout.strip().splitlines():
        name, size, *offs = line.split()
        cls = getattr(capi, name)
        fields = [f for f, _ in cls._fields_]
        assert ctypes.sizeof(cls) == int(size), name
        assert [getattr(cls, f).offset for f in fields] == [int(x) for x in offs], name


def test_missing_library_fails_loudly(tmp_path):
    # no CPU path: without the built library the binding raises instead of
    # falling back to anything
    with pytest.raises(OSError, match="not built"):
        capi.load(str(tmp_path / "libcsc.so"))


@pytest.mark.parametrize("Hz,h,M", [(200, 11, 10), (64, 17, 4), (7, 3, 7), (1000, 8, 0),
                                    (513, 1, 9)])
def test_plan_gives_the_band_schedule_of_the_2d_oracle(lib, Hz, h, M):
    # the 2-D variant cuts rows as the 1-D path cuts time: csc_plan over the
    # Hz rows with atom height h is the 2-D oracle's band schedule
    from oracle import csc2d
    Mo, c, starts = capi.csc_plan(Hz, h, M)
    assert c == csc2d.phase_count(Hz, Mo, h)
    assert [int(x) for x in starts] == [csc2d.band_start(Hz, Mo, m) for m in range(Mo + 1)]


def test_binding_refuses_mismatched_shapes_before_any_call(lib):
    """The C entry points take raw pointers and cannot see array sizes; the
    binding checks shapes first, so a wrong array never reaches a kernel."""
    D = np.zeros((2, 3, 4), np.float32)
    X = np.zeros((3, 64), np.float32)
    Z = np.zeros((2, 61), np.float32)
    with pytest.raises(ValueError):  # Z one column short
        capi.csc_objective_noalloc(D, X, Z[:, :60].copy(), 0.1)
    with pytest.raises(ValueError):  # X with the wrong channel count
        capi.csc_objective_noalloc(D, np.zeros((2, 64), np.float32), Z, 0.1)
    with pytest.raises(ValueError):  # host arrays (the entry point needs device memory)
        capi.csc_objective_noalloc(D, X, Z, 0.1)
    h = capi.Handle()
    h.K, h.P, h.L = 2, 3, 4
    with pytest.raises(ValueError):
        capi.csc_init(h, np.zeros((2, 64), np.float32), 0.1)
    with pytest.raises(ValueError):  # warm start of the wrong size
        capi.csc_init(h, X, 0.1, Z0=np.zeros((2, 60), np.float32))
    with pytest.raises(ValueError):
        capi.csc_init_batch(h, np.zeros((1, 64), np.float32), [64], [0.1])
    h.Tz = 61
    with pytest.raises(ValueError):
        capi.csc_solve(h, 1e-6, 10, np.zeros((2, 60), np.float32))
    with pytest.raises(ValueError):
        capi.csc_objective(h, np.zeros((3, 61), np.float32))
    with pytest.raises(ValueError):
        capi.csc_kkt(h, np.zeros((2, 62), np.float32))
    with pytest.raises(ValueError):
        capi.csc_get_beta(h, np.zeros((2, 60), np.float32))
