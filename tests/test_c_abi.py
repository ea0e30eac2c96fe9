"""The C ABI from C: tests/c/cdmt_example.c includes include/cdmt.h, links
libcdmt.so and the CUDA runtime, and runs both forms through cdmt_execute.
The CPU test compiles and links it; the GPU test runs it and compares its
filterbanks with the FP64 oracle on the input it wrote."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1607_00909_gb300")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    lib = os.path.join(PKG, "libcdmt.so")
    if cc is None or not os.path.exists(lib):
        pytest.skip("no C compiler or no built library")
    cudart = None
    for d in ("lib64", "targets/x86_64-linux/lib", "targets/sbsa-linux/lib", "lib"):
        if os.path.exists(os.path.join(CUDA, d, "libcudart.so")):
            cudart = os.path.join(CUDA, d)
            break
    if cudart is None:
        pytest.skip("no libcudart.so in the CUDA toolkit")
    exe = tmp_path / "cdmt_example"
    subprocess.run([cc, "-std=c11", "-O2", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
                    os.path.join(ROOT, "tests", "c", "cdmt_example.c"), "-o", str(exe), "-L", PKG, "-lcdmt",
                    "-L", cudart, "-lcudart", "-lm", f"-Wl,-rpath,{PKG}", f"-Wl,-rpath,{cudart}"], check=True)
    return exe


def test_c_example_compiles_and_links(tmp_path):
    assert _build(tmp_path).exists()


@pytest.mark.gpu
def test_c_example_runs_and_matches_the_oracle(tmp_path, orc):
    exe = _build(tmp_path)
    o32, o16 = tmp_path / "fb32.bin", tmp_path / "fb16.bin"
    r = subprocess.run([str(exe), str(o32), str(o16)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    nsub, nsamp, nchan, nint, dms, nbin = 2, (1 << 15) + 123, 8, 4, [0.0, 4.0, 8.0], 1 << 14
    x = np.fromfile(str(o32) + ".input", dtype=np.float32).reshape(nsub, nsamp, 4)
    nd = orc.overlap(nsub, 140.0, 0.1953125, dms, nchan, nint, nbin)
    want = orc.filterbank(x, 140.0, 0.1953125, dms, nchan, nint, nbin, nd)
    for path, tol in ((o32, 1e-5), (o16, 2e-3)):
        got = np.fromfile(str(path), dtype=np.float32).reshape(want.shape)
        assert np.max(np.abs(got - want)) / np.mean(want) <= tol, path
