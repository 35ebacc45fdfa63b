"""The C-ABI from a plain C program: tests/abi_client.c is compiled with the
host C compiler against include/hirace.h, linked only to libhirace.so, run on
the GPU, and its report equals the oracle's race set for the same records."""
import os
import re
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_client(oracle_mod, tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2401_04701_gb300 import build as B, tracegen as tg
    exe = str(tmp_path / "abi_client")
    libdir = os.path.dirname(B.LIB)
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-o", exe, os.path.join(ROOT, "tests", "abi_client.c"),
                           "-I", os.path.join(ROOT, "include"), "-L", libdir, "-l:libhirace.so",
                           "-Wl,-rpath," + libdir])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    got = {(int(k), int(w), int(e)) for w, k, e in
           re.findall(r"race word (\d+) kernel (\d+) epoch (\d+)", out.stdout)}
    # the same records, checked by the oracle
    R = tg.RECORD
    rows = [(0, 0, 0, 0, tg.OP_W), (1, 2, 0, 0, tg.OP_R)] + [(0, t, 0, 1, tg.OP_SYNCTHREADS) for t in range(4)] + \
           [(0, 2, 0, 1, tg.OP_R), (1, 1, 0, 1, tg.OP_R)]
    tr = np.zeros(len(rows), R)
    for i, (w, t, wc, bc, op) in enumerate(rows):
        tr[i]["word"], tr[i]["tid"], tr[i]["wc"], tr[i]["bc"], tr[i]["op"] = w, t, wc, bc, op
    want = oracle_mod.race_keys(oracle_mod.bruteforce(tr, 2, 32))
    assert want == {(0, 0, 1)} and got == want, out.stdout
