"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/fsmp.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "fsmp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fsmp_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("fsmp_create", "fsmp_submit", "fsmp_poll", "fsmp_destroy", "fsmp_strerror",
                     "fsmp_run_device"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2403_03156_gb300 import build, fsmp
    path = build.build()
    L = ctypes.CDLL(path)
    for name in declared_entry_points():
        assert hasattr(L, name), name
    assert sorted(fsmp.EXPORTS) == declared_entry_points()


def test_strerror_without_gpu():
    from paper_2403_03156_gb300 import fsmp
    assert fsmp.strerror(fsmp.ERR_BUSY) == "submit queue full"
    assert fsmp.strerror(12345) == "unknown status"


def test_struct_sizes_match_header_layout():
    from paper_2403_03156_gb300 import fsmp
    assert fsmp.SUMMARY_DTYPE.itemsize == 15 * 8 + 14 * 4
    assert fsmp.TRACE_DTYPE.itemsize == 5 * 8 + 4 * 4


def test_binding_refuses_to_run_without_library(monkeypatch, tmp_path):
    from paper_2403_03156_gb300 import fsmp
    monkeypatch.setattr(fsmp, "_lib", None)
    monkeypatch.setattr(fsmp, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        fsmp.load()


def test_params_and_tune_layout_match_the_header(tmp_path):
    """sizeof / offsetof of fsmp_params and fsmp_tune from the C compiler against the ctypes
    mirrors the binding passes across the boundary."""
    import subprocess
    from paper_2403_03156_gb300 import fsmp
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "fsmp.h"\nint main(void) {\n'
                   '  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(fsmp_params), offsetof(fsmp_params, pe_lanes),\n'
                   '         offsetof(fsmp_params, n_mix), offsetof(fsmp_params, mix_sigma), sizeof(fsmp_tune),\n'
                   '         offsetof(fsmp_tune, lanes_per_chain));\n  return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    P, T = fsmp.Params, fsmp.Tune
    assert got == [ctypes.sizeof(P), P.pe_lanes.offset, P.n_mix.offset, P.mix_sigma.offset, ctypes.sizeof(T),
                   T.lanes_per_chain.offset]


def test_create_rejects_bad_mixtures_without_a_gpu():
    """fsmp_create validates before touching a device: G must sum to 1, sigma_e > 0, at most
    FSMP_MAX_MIX components, and a mixture needs the PE-space kernel."""
    from paper_2403_03156_gb300 import fsmp, workloads
    base = dict(workloads.CONFIGS["plain_fp64_256x128"]["params"], n_max=128)
    mix = dict(mix_G=[0.3, 0.7], mix_mu=[1.0, 2.0], mix_sigma=[0.3, 0.5])
    bad = [dict(mix, mix_G=[0.3, 0.6]), dict(mix, mix_sigma=[0.3, 0.0]), dict(mix, kernel=fsmp.KERNEL_SMEM),
           dict(mix, kernel=fsmp.KERNEL_PLAIN), dict(mix, n_mix=9)]
    for extra in bad:
        with pytest.raises(fsmp.FsmpError) as ei:
            fsmp.Context(dict(base, **extra))
        assert ei.value.code == fsmp.ERR_INVALID, extra


def test_library_has_no_undefined_internal_symbols():
    """Every internal function the library calls is defined in it (a source missing from the
    build would otherwise surface only when the library loads on the GPU machine)."""
    import shutil
    import subprocess
    from paper_2403_03156_gb300 import build
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.check_output([nm, "-u", "-C", build.build()]).decode()
    assert not [line for line in out.splitlines() if "fsmp::" in line]


def test_noalloc_checks_params_like_create_without_a_gpu():
    """fsmp_run_device_noalloc applies fsmp_create's parameter checks before it touches a
    device: a CTA of 48 threads (not a whole number of warps), or a non-finite mu_q, is
    refused with FSMP_ERR_INVALID and nothing is launched (this runs on a host with no GPU)."""
    from paper_2403_03156_gb300 import build, fsmp, workloads
    build.build()
    L = fsmp.load()
    base = dict(workloads.CONFIGS["plain_fp64_256x128"]["params"], precision=fsmp.FP32_REFRESH, n_cap=32,
                n_max=128)
    b = fsmp.DeviceBatch()
    b.n_waveforms, b.n_steps, b.n_max_hint = 1, 10, 128
    # stand-in addresses: the call must fail before any pointer is used
    b.samples = b.offsets = b.lambda0 = b.out = 16
    for bad in (dict(threads_per_chain=48), dict(threads_per_chain=2000), dict(mu_q=float("nan"))):
        prm = fsmp.make_params(dict(base, **bad))
        rc = L.fsmp_run_device_noalloc(ctypes.byref(prm), ctypes.byref(b), None)
        assert rc == fsmp.ERR_INVALID, bad
        assert b"checks of fsmp_create" in L.fsmp_last_error(), bad
