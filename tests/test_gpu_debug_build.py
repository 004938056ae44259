"""The bounds-checked debug build (SMAP_DEBUG): every shared-memory row
access and the global sequence / step indices of the step kernels are
checked, a failed check is recorded and the access skipped (nothing traps).
Built here on demand; each case runs in a child process that loads it
through SMAP_LIBRARY and must give exactly the release build's results with
no failed check. The probe shows a check at work on a row index past the
end of a shared array (the check skips the load: nothing is read out of
bounds)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r'''
import json, sys
import numpy as np
from paper_2312_08684_gb300 import Estimator, _binding as abi, workloads as W
out = {}
wl = W.make_range_cv(B=3, T=9, N=40, L=4, dropout=(3, 5))
with Estimator.from_workload(wl) as est:
    path, J = est.run_batch(wl.y)
    out["run_path"] = np.nan_to_num(path, nan=1e30).tolist(); out["run_J"] = J.tolist()
    hist = est.history()
    p2, J2, psi = est.viterbi(hist, wl.y)
    out["vit_J"] = J2.tolist(); out["vit_psi"] = psi.astype(int).tolist()
wl = W.make_clutter_cv(B=4, Tmin=4, Tmax=8, N=70, L=3, uneven_N=(20, 70))
with Estimator.from_workload(wl) as est:
    est.set_variant(3)
    path, J = est.run_batch(wl.y, wl.T, wl.Nseq)
    out["clutter_J"] = J.tolist()
    y = np.ascontiguousarray(wl.y[:, 2])
    xg, hg = est.debug_svgd(3, est.history()[:, 1], est.history()[:, 2], y, 2)
    out["dbg_x"] = xg.tolist()
wl = W.make_ngm1d(B=2, T=6, N=30, L=5)
with Estimator.from_workload(wl) as est:
    path, J = est.pf_run_batch(wl.y)
    out["pf_J"] = J.tolist()
if sys.argv[1] == "debug":
    out["probe_in"] = abi.smap_debug_bounds_probe(16, 15)
    out["probe_out"] = abi.smap_debug_bounds_probe(16, 16)
print(json.dumps(out))
'''


@pytest.fixture(scope="module")
def debug_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_08684_gb300 import build
    return build.build(debug=True)


def _run(which, lib=None):
    env = dict(os.environ)
    env.pop("SMAP_LIBRARY", None)
    if lib:
        env["SMAP_LIBRARY"] = lib
    r = subprocess.run([sys.executable, "-c", CASES, which], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_matches_release_without_failed_checks(debug_lib):
    rel = _run("release")
    dbg = _run("debug", debug_lib)
    for k in rel:
        assert np.array_equal(np.asarray(dbg[k]), np.asarray(rel[k])), k
    # a load inside the array reads it; one row past the end is caught and skipped
    assert dbg["probe_in"] == [1.0, 0, 0]
    assert dbg["probe_out"] == [0.0, 1, 16]


def test_release_build_has_no_probe():
    from paper_2312_08684_gb300 import _binding as abi
    if os.environ.get("SMAP_LIBRARY"):
        pytest.skip("another build is loaded")
    with pytest.raises(abi.SmapError) as e:
        abi.smap_debug_bounds_probe(16, 3)
    assert e.value.status == abi.SMAP_E_UNSUPPORTED
