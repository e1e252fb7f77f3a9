"""Every CUDA kernel of the library waits for its stream predecessor before
it touches memory.

Kernels launched with programmatic serialisation (the setup, and the
captured V-cycle and Arnoldi graphs) may start while the previous kernel is
still running; each must call pdl_wait() (griddepcontrol.wait) before its
first access to data that kernel may write.  Checked on the sources: the
first statement of every __global__ function is pdl_wait()."""
import glob
import os
import re

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1402_4005_gb300", "csrc")

def kernels():
    for path in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        src = open(path).read()
        for m in re.finditer(r"__global__", src):
            line = src[src.rfind("\n", 0, m.start()) + 1:m.start()]
            if line.lstrip().startswith("//"):
                continue
            brace = src.index("{", m.end())
            names = [n for n in re.findall(r"(\w+)\s*\(", src[m.start():brace]) if n != "__launch_bounds__"]
            end = src.index("\n}\n", brace)
            yield os.path.basename(path), names[0], src[brace + 1:end]


def test_every_kernel_waits_first():
    seen = 0
    for fname, name, body in kernels():
        seen += 1
        stmts = [s.strip() for s in body.split(";") if s.strip() and not s.strip().startswith("//")]
        first = re.sub(r"//[^\n]*\n", "", stmts[0] + "\n").strip() if stmts else ""
        assert first == "pdl_wait()", (fname, name, first[:80])
    assert seen >= 90
