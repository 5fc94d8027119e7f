"""Failure detection without a GPU fault: a bounded device wait that runs out must come
back to the host as FK_ETIMEOUT and leave the context usable.

The single-launch conjugate-gradient solver (2-D, D > 1024) synchronises its CTAs
with a grid barrier whose wait is bounded (fk_opts.wait_cycles).  With a bound of one
SM cycle every CTA but the last to arrive gives up at the first barrier, sets the
timeout flag and returns; the CTAs still running see the flag at their next barrier
and return too.  A normal fit on the same stream afterwards must match the oracle.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

fk = pytest.importorskip("paper_2509_02649_b300")


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_cg_barrier_timeout_then_normal_fit():
    n, m, s, lam = 20000, 20, 2.0, 1e-4  # D = 41^2 = 1681 > 1024: the single-launch CG
    x, y = S.wl2_sobolev_2d(n, dtype=np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y).cuda()
    tiny = fk.default_opts(solver=fk.FK_SOLVER_CG, wait_cycles=1)
    with pytest.raises(fk.FkError) as e:
        fk.fk_fit_sobolev(xd, yd, m, s, [lam], 1e-6, "mixed", opts=tiny)
    assert e.value.name == "FK_ETIMEOUT"
    # the context stays usable: the same fit with the default bound, on the same stream
    th = fk.fk_fit_sobolev(xd, yd, m, s, [lam], 1e-6, "mixed", opts=fk.default_opts(solver=fk.FK_SOLVER_CG))
    tho = O.fit(x.astype(np.float64), y.astype(np.float64), m, O.penalty_sobolev(2, m, lam, s))
    assert rel(th[0, 0].cpu().numpy(), tho) <= 1e-5
