"""The C ABI from a C program (tests/c_abi/query_example.c): it builds with a C compiler against
include/taylorgrid.h and the in-tree library, rejects bad arguments without a GPU, and on a GPU gives the
results the Python binding gives for the same points."""
import glob
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2402_14415_gb300")


def cuda_lib_dir():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    for d in [os.path.join(home, "lib64")] + sorted(glob.glob(os.path.join(home, "targets", "*", "lib"))):
        if glob.glob(os.path.join(d, "libcudart.so*")):
            return home, d
    pytest.skip("libcudart not found")


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    if not os.path.exists(os.path.join(PKG, "libtaylorgrid.so")):
        pytest.skip("library not built")
    home, lib = cuda_lib_dir()
    exe = str(tmp_path_factory.mktemp("cabi") / "query_example")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(home, "include"), os.path.join(ROOT, "tests", "c_abi", "query_example.c"),
           "-L", PKG, "-ltaylorgrid", "-L", lib, "-lcudart", "-Wl,-rpath," + PKG, "-Wl,-rpath," + lib, "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


def test_c_program_builds_and_rejects_bad_arguments_without_a_gpu(program):
    r = subprocess.run([program, "host"], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and "host checks ok" in r.stdout, r.stdout + r.stderr


def lcg_points(n):
    """The C program's points: x_{k+1} = 1664525 x_k + 1013904223 (mod 2^32) from 12345, top 24 bits / 2^24."""
    out = np.empty(3 * n, np.float32)
    s = 12345
    for i in range(3 * n):
        s = (s * 1664525 + 1013904223) & 0xFFFFFFFF
        out[i] = np.float32(s >> 8) * np.float32(1.0 / 16777216.0)
    return out.reshape(n, 3)


@pytest.mark.gpu
def test_c_program_matches_the_python_binding(program, tg):
    import torch
    r = subprocess.run([program, "gpu"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    sf, sg, sc = (float(v) for v in r.stdout.split())
    g = tg.tg_create(3, 16, 2, 1, "f32", seed=7, init_std=0.5)
    P = torch.from_numpy(lcg_points(4099)).cuda()
    f = tg.tg_query(g, P)
    grad = torch.zeros(g.n_coefs, device="cuda")
    tg.tg_query_backward(g, P, torch.ones_like(f), grad)
    torch.cuda.synchronize()
    pf, pg = float(f.double().sum()), float(grad.double().sum())
    tg.tg_adam_step(g, grad, lr=1e-2, step=1)
    pc = float(tg.tg_get_coefs(g, which=1).double().sum())
    assert pf == pytest.approx(sf, rel=1e-12, abs=1e-9)        # the same kernel on the same points
    assert pg == pytest.approx(sg, rel=1e-6, abs=1e-6)         # reduction order may differ
    assert pc == pytest.approx(sc, rel=1e-6, abs=1e-6)
