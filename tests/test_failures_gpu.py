"""Failure detection on the GPU path, with every failure made on the host.

No test here faults, traps or hangs the GPU:
* a deadline: lsp_sync with a deadline shorter than the queued work returns
  TIMEOUT and leaves the work queued; a later lsp_sync without a deadline
  returns OK and the result passes oracle parity;
* an allocation failure: lsp_test_fail_allocation makes the context's next
  workspace allocation fail as cudaMalloc would; the call returns OOM and the
  same context then computes correct results;
* the range of the fixed-point phase: a grid whose (t - t_min) f_0 reaches
  2^52 turns is refused through the status word (INVALID_ARG from lsp_sync)
  and its periodogram is NaN instead of silently wrong.
"""
import numpy as np
import pytest

import oracle
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lsp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_1658_gb300 import build, lsp as L
    build.build()
    return L


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_deadline_returns_timeout_then_the_work_completes(lsp):
    from paper_1007_1658_gb300 import synth
    c = synth.corot_382k()
    t, X = _dev(c.t), _dev(c.X)
    with lsp.Context(0) as ctx:
        P = ctx.periodogram(t, X, c.f0, c.df, c.nf)  # ~0.1 s of queued GPU work
        P2 = ctx.periodogram(t, X, c.f0, c.df, c.nf)
        with pytest.raises(lsp.LspError) as e:
            ctx.sync(1e-6)
        assert e.value.status == lsp.ERR_TIMEOUT
        ctx.sync(-1.0)
        got = P.cpu().numpy().astype(np.float64)
        assert np.array_equal(got, P2.cpu().numpy().astype(np.float64))
    rng = np.random.default_rng(5)
    ks = np.unique(np.concatenate([rng.integers(0, c.nf, 48), np.argsort(got)[-16:]]))
    ref = oracle.periodogram_at(c.t, c.X, c.f0 + ks * c.df)
    assert_parity(got[ks], ref, peaks=[], what="after timeout")
    assert np.max(np.abs(got[ks] - ref)) <= 1e-4 * got.max()


@pytest.mark.parametrize("nth", [1, 2, 3])
def test_allocation_failure_leaves_the_context_usable(lsp, nth):
    from paper_1007_1658_gb300 import synth
    c = synth.plain_1k()
    ref = oracle.periodogram(c.t, c.X, c.f0, c.df, c.nf)
    with lsp.Context(0) as ctx:
        ctx.test_fail_allocation(nth)
        with pytest.raises(lsp.LspError) as e:
            ctx.periodogram(_dev(c.t), _dev(c.X), c.f0, c.df, c.nf)
            ctx.sync(30.0)
        assert e.value.status == lsp.ERR_OOM
        P = ctx.periodogram(_dev(c.t), _dev(c.X), c.f0, c.df, c.nf)
        ctx.sync(30.0)
        assert_parity(P.cpu().numpy(), ref, what="after injected OOM")


def test_allocation_failure_in_a_batch_then_the_batch_runs(lsp):
    from paper_1007_1658_gb300 import synth
    pats = synth.noise_batch(n_curves=8, seed=4242, nt_max=3000)
    t_off = torch.from_numpy(pats.t_off).cuda()
    t = _dev(pats.t)
    f0, df, nf = _dev(pats.f0), _dev(pats.df), torch.from_numpy(pats.nf).cuda()
    with lsp.Context(0) as ctx:
        ctx.test_fail_allocation(4)
        with pytest.raises(lsp.LspError) as e:
            ctx.batch(t_off, t, f0, df, nf, seed=11, n_real=2)
        assert e.value.status == lsp.ERR_OOM
        m1, a1 = ctx.batch(t_off, t, f0, df, nf, seed=11, n_real=2)
        ctx.sync(60.0)
    with lsp.Context(0) as ref_ctx:
        m2, a2 = ref_ctx.batch(t_off, t, f0, df, nf, seed=11, n_real=2)
        ref_ctx.sync(60.0)
    assert torch.equal(m1, m2) and torch.equal(a1, a2)


def test_fixed_point_phase_range_is_refused(lsp):
    from paper_1007_1658_gb300 import synth
    c = synth.plain_1k()
    f0 = 1e15  # (t - t_min) f_0 up to 1e17 turns, beyond 2^52
    with lsp.Context(0) as ctx:
        P = ctx.periodogram(_dev(c.t), _dev(c.X), f0, c.df, 64)
        with pytest.raises(lsp.LspError) as e:
            ctx.sync(30.0)
        assert e.value.status == lsp.ERR_INVALID_ARG
        assert torch.isnan(P).all()
        # host pointers: the call blocks and reports it itself
        with pytest.raises(lsp.LspError) as e:
            ctx.periodogram(c.t, c.X, c.f0, 1e14, 64)
        assert e.value.status == lsp.ERR_INVALID_ARG
        # the context still works, and a grid just inside the range passes
        P = ctx.periodogram(_dev(c.t), _dev(c.X), c.f0, c.df, c.nf)
        ctx.sync(30.0)
        assert_parity(P.cpu().numpy(), oracle.periodogram(c.t, c.X, c.f0, c.df, c.nf), what="after refusal")
