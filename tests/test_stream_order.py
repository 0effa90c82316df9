"""Host-side check of the library's stream discipline (no GPU needed).

Handles may own non-blocking streams (SE_MESH_NONBLOCKING_STREAM, and every mesh the solve server
builds).  The legacy default stream does not order with such streams, so a synchronous
cudaMemcpy/cudaMemset issued during set-up could still be in flight when a set-up kernel on the
handle's stream reads its target.  Every upload, symbol write and zero fill in the CUDA sources
must therefore name a stream (cudaMemcpyAsync / cudaMemsetAsync, usually through h2d / dzero).
"""
import pathlib
import re

import pytest

CSRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2110_07663_gb300" / "csrc"


def _calls(text, name):
    """Yield the argument text of every call `name(` ... `)` in `text` (nested parentheses kept)."""
    for m in re.finditer(r"\b" + re.escape(name) + r"\s*\(", text):
        depth, i = 1, m.end()
        while depth and i < len(text):
            depth += {"(": 1, ")": -1}.get(text[i], 0)
            i += 1
        yield m.start(), text[m.end():i - 1]


def _sources():
    files = sorted(CSRC.glob("*.cu")) + sorted(CSRC.glob("*.h"))
    assert files, "CUDA sources not found"
    return files


@pytest.mark.parametrize("name", ["cudaMemset", "cudaMemcpyToSymbol", "cudaMemset2D", "cudaMemset3D"])
def test_no_unordered_device_writes(name):
    bad = []
    for f in _sources():
        text = f.read_text()
        for pos, _ in _calls(text, name):
            bad.append(f"{f.name}:{text.count(chr(10), 0, pos) + 1}")
    assert not bad, f"{name} on the legacy stream: {bad}"


def test_no_synchronous_uploads():
    bad = []
    for f in _sources():
        text = f.read_text()
        for pos, args in _calls(text, "cudaMemcpy"):
            if "cudaMemcpyDeviceToHost" not in args:
                bad.append(f"{f.name}:{text.count(chr(10), 0, pos) + 1}")
    assert not bad, f"synchronous cudaMemcpy that writes device memory: {bad}"


def test_the_check_sees_a_planted_upload(tmp_path):
    """The scanner itself: a synchronous upload and a memset in a planted source are found."""
    text = "int f(double* d, const double* h) {\n  cudaMemcpy(d, h, 8, cudaMemcpyHostToDevice);\n" \
           "  cudaMemset(d, 0, 8);\n  cudaMemcpyAsync(d, h, 8, cudaMemcpyHostToDevice, s);\n}\n"
    ups = [a for _, a in _calls(text, "cudaMemcpy") if "cudaMemcpyDeviceToHost" not in a]
    sets = list(_calls(text, "cudaMemset"))
    assert len(ups) == 1 and len(sets) == 1
