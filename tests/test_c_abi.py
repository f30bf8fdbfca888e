"""The C ABI from a plain C program (tests/c_abi/sp2_lattice.c): it compiles against
include/gbe.h with -Wall -Wextra -Werror and links against the in-tree libgbe.so; without a
GPU it stops at gbe_create with an error (no CPU fallback); on the GPU it builds H, the
|H^2| graph, the partition, runs SP2 and assembles D into host buffers, and its D equals,
bit for bit, what the Python binding computes on the same input."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi", "sp2_lattice.c")
gbe = pytest.importorskip("paper_1603_00937_gb300")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    if not os.path.exists(gbe.LIB_PATH):
        from paper_1603_00937_gb300 import build
        build.build()
    libdir = os.path.dirname(gbe.LIB_PATH)
    out = str(tmp_path_factory.mktemp("c_abi") / "sp2_lattice")
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I" + os.path.join(ROOT, "include"), SRC,
                        "-L" + libdir, "-lgbe", "-Wl,-rpath," + libdir, "-o", out], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def write_input(path, w):
    with open(path, "wb") as f:
        np.array([w["pos"].shape[0]], np.int64).tofile(f)
        np.asarray(w["box"], np.float64).tofile(f)
        np.ascontiguousarray(w["pos"], np.float64).tofile(f)
        np.ascontiguousarray(w["onsite"], np.float64).tofile(f)


def read_output(path):
    with open(path, "rb") as f:
        iters, stop = np.fromfile(f, np.int32, 2)
        eps = np.fromfile(f, np.float64, 2)
        n, width = np.fromfile(f, np.int64, 2)
        col = np.fromfile(f, np.int32, n * width).reshape(n, width)
        val = np.fromfile(f, np.float64, n * width).reshape(n, width)
    return int(iters), int(stop), eps, col, val


def test_c_program_links(exe):
    assert os.access(exe, os.X_OK)


def test_c_program_without_gpu_fails_loudly(exe, tmp_path):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    w = synth.lattice(4, seed=0)
    write_input(tmp_path / "in.bin", w)
    r = subprocess.run([exe, str(tmp_path / "in.bin"), str(tmp_path / "out.bin"), "1e-5", "2", "1"],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 2 and "gbe_create" in r.stderr, (r.returncode, r.stderr)
    assert not (tmp_path / "out.bin").exists()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [gbe.PREC_FP64, gbe.PREC_FP16X6, gbe.PREC_FP64TC])
def test_c_program_matches_binding(exe, tmp_path, prec):
    import torch
    w = synth.lattice(8, seed=0)
    write_input(tmp_path / "in.bin", w)
    r = subprocess.run([exe, str(tmp_path / "in.bin"), str(tmp_path / "out.bin"), "1e-5", "4", str(prec)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    iters, stop, eps, col, val = read_output(tmp_path / "out.bin")
    ctx = gbe.Context(0)
    st = gbe.sites(w["pos"], w["onsite"], w["box"])
    H = gbe.build_hamiltonian(ctx, st)
    S = gbe.build_graph(ctx, H.csr(), gbe.GRAPH_H2_THRESH, thresh=1e-5)
    parts = gbe.partition(ctx, S, gbe.PART_SPATIAL_CELLS, ncell=(4, 4, 4), site_struct=st)
    X, rep = gbe.sp2_submatrices(ctx, H.csr(), parts, gbe.sp2_params(w["pos"].shape[0] / 2.0, prec=prec))
    n, width = gbe.assemble_width(ctx, X, parts)
    col_b = np.empty((n, width), np.int32)
    val_b = np.empty((n, width), np.float64)
    gbe.assemble_D(ctx, X, parts, col_b, val_b)
    torch.cuda.synchronize()
    assert iters == rep["iters"] and tuple(eps) == tuple(rep["eps"])
    assert np.array_equal(col, col_b) and np.array_equal(val, val_b)
