"""The C ABI from plain C: tests/capi_example.c includes only include/sdm.h and links libsdm.so.

* (CPU) it compiles as strict C11 with every warning an error and links against the library, so
  the header is a C header (no C++ constructs leak through) and every call the program makes is
  exported;
* (GPU) run on a Golovin box and on a gravitational box, its state after 12 steps equals the
  oracle's bit for bit, and its step statistics agree.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import oracle
from paper_2101_06318_b300 import build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "capi_example.c")


def _compile(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:  # pragma: no cover
        pytest.skip("no C compiler")
    lib = build.build()
    exe = str(tmp_path / "capi_example")
    libdir = os.path.dirname(lib)
    cmd = [cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-O2", "-I", os.path.join(ROOT, "include"),
           SRC, "-o", exe, "-L", libdir, "-lsdm", "-Wl,-rpath," + libdir]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


def test_c_program_compiles_and_links(tmp_path):
    exe = _compile(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True)     # no arguments: usage, exit 1
    assert r.returncode == 1 and "usage" in r.stderr


@pytest.mark.gpu
@pytest.mark.parametrize("box", ["golovin", "gravitational"])
def test_c_program_steps_bitexact(tmp_path, box):
    exe = _compile(tmp_path)
    s = inputs.golovin_box() if box == "golovin" else inputs.gravitational_box(n_sd=1 << 16)
    n, steps, seed = len(s["xi"]), 12, 2021
    kid = int(s["kernel_id"][0])
    src, dst = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(src, "wb") as f:
        f.write(struct.pack("<Q", n))
        f.write(s["xi"].astype("<u8").tobytes())
        f.write(s["v"].astype("<f8").tobytes())
        f.write(struct.pack("<dddQ", float(s["dv"][0]), float(s["golovin_b"]), float(s["dt"]), seed))
    r = subprocess.run([exe, str(src), str(dst), str(steps), str(kid)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    raw = open(dst, "rb").read()
    (m,) = struct.unpack_from("<Q", raw, 0)
    assert m == n
    xi = np.frombuffer(raw, "<u8", n, 8)
    v = np.frombuffer(raw, "<f8", n, 8 + 8 * n)
    n_pairs, n_coll, n_rem = struct.unpack_from("<QQQ", raw, 8 + 16 * n)
    o = oracle.System(s["xi"], s["v"], s["cell_start"], s["dv"], s["kernel_id"], s["golovin_b"], "prp")
    ost = o.run(s["dt"], seed, 0, steps)
    assert np.array_equal(xi, o.xi)
    assert np.array_equal(v.view(np.uint64), o.attr[0].view(np.uint64))
    assert n_coll == ost["n_collisions"] > 0 and n_rem == ost["n_removed"]
    assert n_pairs == ost["n_pairs"]
