"""The bounds-checked build (libfk_checked.so, FK_CHECKED): the stand-in for a memory
checker.  Its kernels test the data-dependent indices of the spreading paths (cells
named by partition records, list links, grid nodes, bucket slots) and return
FK_EINTERNAL instead of making an access that fails a test.  Here the parity cases of
each spreading path run in a fresh process on that library and must match the oracle
with no check failing (a failed check would raise FK_EINTERNAL)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, "@ROOT@")
import numpy as np, torch
import paper_2509_02649_b300 as fk
import oracle as O, synthetic as S
assert fk.lib()._name.endswith("libfk_checked.so"), fk.lib()._name
rel = lambda a, b: float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))
# 2-D one-pass partition + register accumulation (n % 4 == 0) and the exact partition (odd n)
for n in (40000, 40003):
    x, y = S.wl2_sobolev_2d(n, dtype=np.float32)
    T, b = fk.fk_build_system(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 12, 1e-6, "mixed")
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    assert rel(T.cpu().numpy(), O.moments(x64, 12)) <= 1e-5
    assert rel(b.cpu().numpy()[0], O.rhs(x64, y64, 12)) <= 1e-5
# 1-D fixed-point spreader, many channels
x = S.uniform_points(30000, 1, 7).astype(np.float32)
c = np.stack([S.noise(30000, 1.0, 7, k) for k in range(5)]).astype(np.float32)
out = fk.fk_type1(torch.from_numpy(x).cuda(), torch.from_numpy(c).cuda(), 40, 1e-6, "mixed").cpu().numpy()
ref = O.type1(x.astype(np.float64), c.astype(np.float64), 40)
assert max(rel(out[k], ref[k]) for k in range(5)) <= 1e-5
# additive pair blocks from the row-owner partition
X, yv = S.wl4_additive(16000, d=4, dtype=np.float32)
th = fk.fk_fit_additive(torch.from_numpy(X).cuda(), torch.from_numpy(yv).cuda(), 10, [1e-3], 1e-6, "mixed")
tho = O.fit_additive(X.astype(np.float64), yv.astype(np.float64), 10, 1e-3).reshape(4, 21)
keep = lambda t: np.concatenate([np.delete(t, 10, axis=1).ravel(), [t[:, 10].sum()]])
assert rel(keep(th[0, 0].cpu().numpy()), keep(tho)) <= 1e-5
print("checked build ok")
""".replace("@ROOT@", ROOT)


def test_checked_build_runs_the_spreading_paths_clean():
    lib = os.path.join(ROOT, "paper_2509_02649_b300", "libfk_checked.so")
    if not os.path.exists(lib):
        pytest.skip("libfk_checked.so is not built")
    env = dict(os.environ, FK_CHECKED="1")
    out = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert "checked build ok" in out.stdout
