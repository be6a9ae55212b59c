"""A plain C program (tests/c_consumer.c) built against include/ch.h and
linked to libch.so: it must compile and link on the CPU, and on the GPU run
ch_reduce -> ch_chain -> ch_hull and ch_chain_noalloc on Fig. 1's points
(Section 2.1) and on a larger seeded set, printing L, both chains and the
hull, which are checked against the paper's printed values and the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1505_00914_gb300 import _build, synth
from _golden import read
from test_oracle import _fig1_points

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime.h")):
            return c
    pytest.skip("CUDA toolkit headers not found")


def build_consumer(out_dir):
    if not shutil.which("cc") and not shutil.which("gcc"):
        pytest.skip("no C compiler")
    lib = _build.build()
    cuda = _cuda_home()
    libdirs = [d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib")) if os.path.isdir(d)]
    exe = os.path.join(out_dir, "c_consumer")
    cmd = [shutil.which("cc") or "gcc", "-std=c99", "-O1", "-Wall", "-Werror",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
           os.path.join(HERE, "c_consumer.c"), "-o", exe, lib,
           "-Wl,-rpath," + os.path.dirname(lib)]
    for d in libdirs:
        cmd += ["-L", d, "-Wl,-rpath," + d]
    cmd += ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, " ".join(cmd) + "\n" + r.stdout + r.stderr
    return exe


def test_c_consumer_compiles_and_links(tmp_path):
    exe = build_consumer(str(tmp_path))
    assert os.path.exists(exe)


def _run(exe, P, p, tmp_path):
    inp = os.path.join(str(tmp_path), f"pts_{p}.txt")
    with open(inp, "w") as f:
        f.write(f"{P.shape[0]} {p}\n")
        np.savetxt(f, P, fmt="%d")
    r = subprocess.run([exe, inp], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr
    out = {}
    for line in r.stdout.splitlines():
        k, *v = line.split()
        out.setdefault(k, []).append([int(x) for x in v])
    assert out.get("ok") == [[]]
    arr = lambda k, w: np.asarray(out.get(k, []), np.int64).reshape(-1, w)
    return {"L": arr("L", 3)[:, 1:], "lower": arr("lower", 2), "upper": arr("upper", 2),
            "nlower": arr("nlower", 2), "nupper": arr("nupper", 2), "hull": arr("hull", 2),
            "status": out["status"][0][0]}


@pytest.mark.gpu
def test_c_consumer_fig1_and_seeded_set(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = build_consumer(str(tmp_path))
    # Fig. 1: the paper's printed L and the pentagon
    keys, L = read("fig1_L.txt")
    hk, H = read("fig1_hull.txt")
    o = _run(exe, _fig1_points(seed=1), keys["p"], tmp_path)
    assert o["status"] == 0
    np.testing.assert_array_equal(o["L"], L)
    np.testing.assert_array_equal(o["hull"], H)
    assert o["hull"].shape[0] == hk["count"]
    xs = np.arange(1, keys["p"] + 1)
    np.testing.assert_array_equal(o["lower"], np.stack([xs, L[:, 0]], 1))
    np.testing.assert_array_equal(o["upper"], np.stack([xs, L[:, 1]], 1))
    np.testing.assert_array_equal(o["nlower"], o["lower"])
    np.testing.assert_array_equal(o["nupper"], o["upper"])
    # a seeded disc of 200,000 points at p = 5000 against the oracle
    p = 5000
    P = synth.points("disc", 200_000, p, seed=77)
    o = _run(exe, P, p, tmp_path)
    assert o["status"] == 0
    Lo = oracle.reduce(P, p)
    np.testing.assert_array_equal(o["L"], Lo)
    lo, up = oracle.chain(Lo)
    for k, ref in (("lower", lo), ("upper", up), ("nlower", lo), ("nupper", up)):
        np.testing.assert_array_equal(o[k], ref)
    np.testing.assert_array_equal(o["hull"], oracle.hull_chain(Lo))
