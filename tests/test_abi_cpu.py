"""The C-ABI library builds, loads and exports every symbol include/fpca.h declares.

No compute call is made here (no GPU in this environment).
"""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fpca.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fpca_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1510_04439_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def test_header_declares_the_path_entry_points():
    fns = declared_functions()
    for name in ("fpca_bin_mean", "fpca_smooth_mean", "fpca_bin_cov", "fpca_smooth_cov_project",
                 "fpca_rproj_eig"):
        assert name in fns


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, f"not exported: {missing}"


def test_binding_loads_and_knows_every_symbol(libpath):
    from paper_1510_04439_gb300 import binding
    lib = binding.load(libpath)
    for name in declared_functions():
        assert hasattr(lib, name)
    assert sorted(binding.SYMBOLS) == sorted(
        f for f in declared_functions() if f in binding.SYMBOLS)
    assert set(declared_functions()) <= set(binding.SYMBOLS) | set()


def test_create_without_gpu_fails_cleanly(libpath):
    """With no device, fpca_create returns an error status instead of crashing."""
    import ctypes
    from paper_1510_04439_gb300 import binding
    lib = binding.load(libpath)
    h = ctypes.c_void_p()
    st = lib.fpca_create(ctypes.byref(h), 0, None)
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        assert st in (binding.OK, binding.E_UNSUPPORTED)
        if st == binding.OK:
            lib.fpca_destroy(h)
    else:
        assert st == binding.E_CUDA
        assert not h.value


def test_null_context_is_rejected(libpath):
    from paper_1510_04439_gb300 import binding
    lib = binding.load(libpath)
    assert lib.fpca_sync(None) == binding.E_INVALID_ARG
    assert lib.fpca_bin_mean(None, None, None, None, None, None, None) == binding.E_INVALID_ARG


def test_cov_factor_bytes_is_a_host_function(libpath):
    """The factor size needs no device: R/sqrt(n) in FP32 (P x n_pad) and in BF16 twice
    (n_pad x p_pad, p_pad x n_pad), plus the P node sums, each 256-byte aligned."""
    from paper_1510_04439_gb300 import binding
    lib = binding.load(libpath)

    def size(m, n):
        return int(lib.fpca_cov_factor_bytes(binding.Grid.of(m), n))

    def expect(m, n):
        P = m[0] * m[1] * m[2]
        n_pad = (n + 127) // 128 * 128
        p_pad = 128 * ((m[0] + 3) // 4) * ((m[1] + 3) // 4) * ((m[2] + 7) // 8)
        total = 0
        for b in (4 * P * n_pad, 2 * n_pad * p_pad, 2 * p_pad * n_pad, 4 * P):
            total += (b + 255) // 256 * 256
        return total

    for m, n in [((32, 32, 32), 2000), ((6, 5, 12), 45), ((8, 8, 8), 1)]:
        assert size(m, n) == expect(m, n)
    assert size((16, 16), 10) == 0          # not a 3-D grid


def test_bw_param_count_is_the_oracle_layout(libpath):
    """The network's parameter count needs no device and equals the oracle's layout:
    for each layer of 32 -> 256 -> 256 -> 256 -> 6, fan_in x fan_out weights then fan_out
    biases."""
    from oracle import mlp as om
    from paper_1510_04439_gb300 import binding
    lib = binding.load(libpath)
    n = int(lib.fpca_bw_param_count())
    assert n == om.param_count()
    assert n == sum(fi * fo + fo for fi, fo in [(32, 256), (256, 256), (256, 256), (256, 6)])
