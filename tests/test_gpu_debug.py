"""The debug build (libdfilt_debug.so, -DDFILT_DEBUG): the decoupled path's device-side
index checks on a GPU, without touching memory outside any buffer.

The debug library runs in a child process (DFILT_LIBRARY=debug picks it at import).  It
takes the ragged case of test_gpu_hi.test_decoupled_ragged (every state bucket, spans
of two tiles, empty channels) and must give
  - with no limit: status DFILT_OK and outputs bit-identical to the release library's
    (the checks pass and change no arithmetic; the release outputs are checked against
    the FP64 oracle by that test);
  - with dfilt_debug_set_limit below the batch's length: DFILT_ERR_BOUNDS (the checks
    fail on the tiles and spans past the limit, and those are skipped -- every buffer
    is still the caller's full, valid one, so nothing out of bounds is ever addressed);
  - with the limit removed again: DFILT_OK and the same outputs as the first call.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2511_14390_gb300 import dfilt, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
NAMES = ("y", "gx", "gb", "ga", "gz")


def make_case():
    w = inputs.make_ragged(B=30, T_range=(1, 70000), M_range=(1, 64), seed=841)
    lens = np.diff(w.offsets)
    lens[[4, 11]] = 0
    offs = np.zeros_like(w.offsets)
    offs[1:] = np.cumsum(lens)
    w.x = np.concatenate([w.x[w.offsets[i]:w.offsets[i] + lens[i]] for i in range(w.B)])
    w.gy = np.concatenate([w.gy[w.offsets[i]:w.offsets[i] + lens[i]] for i in range(w.B)])
    w.offsets = offs
    return w


def run_case(w):
    """forward + backward through the loaded library; outputs and the status word"""
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    o = dfilt.make_opts(algo="chunked", path="decoupled", span_tiles=2)
    dx, dgy = dev(w.x), dev(w.gy)
    doffs, dMs, dNs = dev(w.offsets), dev(w.Ms), dev(w.Ns)
    db, da, dzi = dev(w.b), dev(w.a), dev(w.zi)
    y, saved = dfilt.dfilt_forward_ragged(dx, doffs, dMs, dNs, db, da, dzi, opts=o)
    g = dfilt.dfilt_backward_ragged(dgy, dx, None, doffs, dMs, dNs, db, da, dzi, saved, opts=o)
    st = dfilt.dfilt_sync_status()
    return [t.cpu().numpy() for t in (y, *g)], st


def child(out_path):
    """Runs under DFILT_LIBRARY=debug: no limit, a limit, no limit again."""
    assert dfilt.dfilt_debug_build()
    w = make_case()
    total = int(w.offsets[-1])
    res0, st0 = run_case(w)
    dfilt.dfilt_debug_set_limit(total - 20000)
    _, st1 = run_case(w)
    dfilt.dfilt_debug_set_limit(0)
    res2, st2 = run_case(w)
    np.savez(out_path, st=np.array([st0, st1, st2]), total=total,
             **{f"a_{n}": v for n, v in zip(NAMES, res0)},
             **{f"c_{n}": v for n, v in zip(NAMES, res2)})


def test_debug_library_checks(tmp_path):
    from paper_2511_14390_gb300 import build as pkg_build
    pkg_build.build_debug()
    assert not dfilt.dfilt_debug_build()   # this process runs the release library
    w = make_case()
    ref, st = run_case(w)
    assert st == 0
    out = str(tmp_path / "debug_child.npz")
    env = dict(os.environ, DFILT_LIBRARY="debug")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), out], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    d = np.load(out)
    try:
        st0, st1, st2 = (int(v) for v in d["st"])
        assert int(d["total"]) > 20000
        assert st0 == 0, dfilt.STATUS.get(st0, st0)
        assert st1 == 7, dfilt.STATUS.get(st1, st1)      # DFILT_ERR_BOUNDS
        assert st2 == 0, dfilt.STATUS.get(st2, st2)
        for n, v in zip(NAMES, ref):
            assert np.array_equal(d[f"a_{n}"], v), n      # debug == release, bit for bit
            assert np.array_equal(d[f"c_{n}"], v), n      # and again after the limit
    finally:
        d.close()


if __name__ == "__main__":
    child(sys.argv[1])
