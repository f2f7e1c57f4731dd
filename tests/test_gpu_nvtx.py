"""NVTX ranges: the library names the phases of a solve and of the batch
engine (header-only NVTX v3).  A small injection library
(`tests/nvtx_recorder.c`, loaded by NVTX through NVTX_INJECTION64_PATH)
records every range push and pop; the CPU test checks the recorder on a
plain C program, the GPU test runs a solve and a batch in a fresh process
and checks the library's ranges and their nesting."""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cuda_include():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(cand))), "include")
            if os.path.exists(os.path.join(inc, "nvtx3", "nvToolsExt.h")):
                return inc
    pytest.skip("NVTX v3 headers not found")


def _build_recorder(tmp_path):
    inc = _cuda_include()
    out = str(tmp_path / "libnvtx_recorder.so")
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", f"-I{inc}",
                           os.path.join(HERE, "nvtx_recorder.c"), "-o", out, "-lpthread"])
    return out, inc


def _events(log):
    with open(log) as fh:
        return [ln.rstrip("\n") for ln in fh if ln.strip()]


def _tree(events, names):
    """Nesting of the ranges whose names are in `names`: a list of
    (depth, name), with pushes and pops checked to balance."""
    stack, out = [], []
    for ev in events:
        if ev.startswith("push "):
            stack.append(ev[5:])
            if stack[-1] in names:
                out.append((sum(1 for s in stack[:-1] if s in names), stack[-1]))
        else:
            assert ev == "pop" and stack, events
            stack.pop()
    assert not stack, f"unbalanced ranges: {stack}"
    return out


def test_recorder_sees_pushes_and_pops(tmp_path):
    """The recorder itself, on a C program that opens two nested ranges."""
    rec, inc = _build_recorder(tmp_path)
    src = tmp_path / "probe.c"
    src.write_text(textwrap.dedent("""
        #include <nvtx3/nvToolsExt.h>
        int main(void) {
            nvtxRangePushA("outer");
            nvtxRangePushA("inner");
            nvtxRangePop();
            nvtxRangePop();
            return 0;
        }
    """))
    exe = str(tmp_path / "probe")
    subprocess.check_call(["gcc", "-O1", f"-I{inc}", str(src), "-o", exe, "-ldl"])
    log = str(tmp_path / "nvtx.log")
    env = dict(os.environ, NVTX_INJECTION64_PATH=rec, PDOT_NVTX_LOG=log)
    subprocess.check_call([exe], env=env)
    assert _events(log) == ["push outer", "push inner", "pop", "pop"]


_CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import torch
    from paper_2407_19689_gb300 import instances as I, pdot
    ins = I.points_instance(40, 56, 11)
    s = pdot.Solver(device=0)
    sol = s.solve(torch.tensor(ins.C, dtype=torch.float32, device="cuda:0"), ins.f, ins.g, tol=1e-4)
    assert sol.status == pdot.OK, sol.result
    s.close()
    b = pdot.BatchSolver(device=0)
    for k in range(2):
        j = I.points_instance(30 + 7 * k, 45, 20 + k)
        b.submit(torch.tensor(j.C, dtype=torch.float32, device="cuda:0"), j.f, j.g, tol=1e-4)
    done = b.run()
    assert len(done) == 2
    b.close()
""")


@pytest.mark.gpu
def test_solve_and_batch_ranges(tmp_path):
    """A solve opens pdot_solve with its phases autotune, start, chunks and
    result nested inside, in that order; the batch engine's polls open
    pdot_poll with retire / admit / launch chunk inside."""
    from paper_2407_19689_gb300 import pdot
    pdot.load(build_if_missing=True)
    rec, _ = _build_recorder(tmp_path)
    log = str(tmp_path / "nvtx.log")
    env = dict(os.environ, NVTX_INJECTION64_PATH=rec, PDOT_NVTX_LOG=log)
    subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT)], env=env, check=True, timeout=300)
    names = {"pdot_solve", "autotune", "start", "chunks", "result", "pdot_batch_submit", "pdot_poll", "retire",
             "admit", "launch chunk"}
    tree = _tree(_events(log), names)
    solve = tree[: tree.index((0, "pdot_batch_submit"))]
    assert solve == [(0, "pdot_solve"), (1, "autotune"), (1, "start"), (1, "chunks"), (1, "result")]
    batch = tree[len(solve):]
    assert batch.count((0, "pdot_batch_submit")) == 2
    polls = [t for t in batch if t == (0, "pdot_poll")]
    assert polls
    inner = {name for depth, name in batch if depth == 1}
    assert {"retire", "admit", "launch chunk"} <= inner
    assert all(d <= 1 for d, _ in tree)
