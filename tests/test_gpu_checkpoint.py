"""Checkpoint / resume of a device-resident cell (mp_checkpoint, mp_resume)
and the reset-to-initial-state path: a run resumed from a checkpoint taken
between load increments, and a run after mp_rve_reset, equal an
uninterrupted run from a fresh cell bit for bit."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2409_10774_gb300 as M
    return M.Context(0)


def _problem():
    return W.workload_batch(count=1, sizes=(16,), n_steps=6, tol=1e-6, seed=W.seed_for(3) + 77)[0]


def _same(a, b):
    assert a["steps_done"] == b["steps_done"] and a["failed_step"] == b["failed_step"]
    for k in ("T", "M", "Eavg", "Gavg", "P", "Q", "Teq", "Meq", "err", "iters"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("e", "g", "t", "m", "p", "q"):
        assert np.array_equal(a["final"][k], b["final"][k]), k


@pytest.mark.parametrize("precision", [0, 1])
def test_resume_equals_uninterrupted_run(ctx, precision):
    import paper_2409_10774_gb300 as M
    p = _problem()
    a = M.Rve(ctx, p, precision=precision)
    a.run(2)
    image = a.checkpoint()
    a.run(4)
    ra = a.results(fields=True)
    a.close()
    b = M.Rve(ctx, p, precision=precision)
    b.resume(image)
    assert b.steps_done == 2
    b.run(4)
    rb = b.results(fields=True)
    b.close()
    assert ra["steps_done"] == 6
    _same(ra, rb)


def test_resume_refuses_another_problem(ctx):
    import paper_2409_10774_gb300 as M
    from paper_2409_10774_gb300 import binding as B
    p = _problem()
    a = M.Rve(ctx, p, precision=1)
    a.run(1)
    image = a.checkpoint()
    a.close()
    for other, prec in ((dict(p, tol=1e-7), 1), (p, 0)):
        c = M.Rve(ctx, other, precision=prec)
        with pytest.raises(B.MicropolarError) as ei:
            c.resume(image)
        assert ei.value.status == 1
        c.close()
    d = M.Rve(ctx, p, precision=1)
    with pytest.raises(B.MicropolarError):
        d.resume(image[:100])
    d.close()


def test_reset_equals_fresh_cell(ctx):
    import paper_2409_10774_gb300 as M
    p = _problem()
    a = M.Rve(ctx, p, precision=1)
    a.run(3)
    a.reset()
    a.run(3)
    ra = a.results(fields=True)
    a.close()
    b = M.Rve(ctx, p, precision=1)
    b.run(3)
    rb = b.results(fields=True)
    b.close()
    _same(ra, rb)
