"""Canary-padded outputs: every entry point writes exactly its output range.

Each output is a view into a larger buffer whose pads (and, for the batches,
the slack that P_off leaves between curves) hold a NaN bit pattern that no
kernel writes; after the call and a sync the pads must hold it bit for bit.
Sizes are ragged (N_t not a multiple of the sample tile, N_f not a multiple
of a strip or of a CTA's block of frequencies), and both the direct-write
(one N_t chunk) and the split-plus-finalize paths run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lsp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_1658_gb300 import build, lsp as L
    build.build()
    return L


CANARY = np.int32(0x7FA5A5A5)  # a quiet NaN with a payload
PAD = 1024  # floats on each side; keeps the 16-byte alignment of the buffer


def _padded(n, device="cuda"):
    buf = torch.full((n + 2 * PAD,), int(CANARY), dtype=torch.int32, device=device)
    return buf, buf.view(torch.float32)[PAD:PAD + n]


def _pads_intact(buf, n):
    b = buf.cpu().numpy()
    return np.all(b[:PAD] == CANARY) and np.all(b[PAD + n:] == CANARY)


def _curve(n, seed):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, 60.0, n))
    X = rng.normal(size=n) + np.sin(2 * np.pi * 0.41 * t)
    dy = np.exp(rng.uniform(np.log(0.3), np.log(2.0), n))
    return t, X, dy


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("mode,phase", [(1, 0), (2, 0), (3, 0), (4, 0), (1, 1)])
@pytest.mark.parametrize("n_t,n_f", [(3001, 4097), (130, 77), (60000, 1001)])
def test_periodogram_writes_only_its_range(lsp, mode, phase, n_t, n_f):
    t, X, _ = _curve(n_t, 11)
    ctx = lsp.Context(0, sincos_mode=mode, phase_mode=phase)
    buf, P = _padded(n_f)
    ctx.periodogram(_dev(t), _dev(X), 0.01, 0.013, n_f, out=P)
    ctx.sync(60.0)
    assert _pads_intact(buf, n_f)
    assert torch.isfinite(P).all()
    ctx.close()


@pytest.mark.parametrize("n_t,n_f", [(3001, 4097), (60000, 1001)])
def test_floating_mean_and_press_rybicki_write_only_their_range(lsp, n_t, n_f):
    t, X, dy = _curve(n_t, 12)
    ctx = lsp.Context(0)
    buf, P = _padded(n_f)
    ctx.periodogram_gls(_dev(t), _dev(X), 0.01, 0.013, n_f, dy=_dev(dy), out=P)
    ctx.sync(60.0)
    assert _pads_intact(buf, n_f) and torch.isfinite(P).all()
    buf, P = _padded(n_f)
    ctx.press_rybicki(_dev(t), _dev(X), 0.013, 0.013, n_f, out=P)
    ctx.sync(60.0)
    assert _pads_intact(buf, n_f) and torch.isfinite(P).all()
    ctx.close()


def test_host_output_writes_only_its_range(lsp):
    t, X, _ = _curve(3001, 13)
    n_f = 4097
    buf = np.full(n_f + 2 * PAD, CANARY, dtype=np.int32)
    P = buf.view(np.float32)[PAD:PAD + n_f]
    ctx = lsp.Context(0)
    ctx.periodogram(t, X, 0.01, 0.013, n_f, out=P)
    assert np.all(buf[:PAD] == CANARY) and np.all(buf[PAD + n_f:] == CANARY)
    assert np.all(np.isfinite(P))
    ctx.close()


def test_noalloc_writes_only_its_range(lsp):
    t, X, _ = _curve(3001, 14)
    n_f = 4097
    buf, P = _padded(n_f)
    lsp.periodogram_noalloc(_dev(t), _dev(X), 0.01, 0.013, n_f, P)
    torch.cuda.synchronize()
    assert _pads_intact(buf, n_f) and torch.isfinite(P).all()


def _batch_with_slack(n_curves=9, seed=21):
    from paper_1007_1658_gb300 import synth
    b = synth.noise_batch(n_curves=n_curves, seed=seed, nt_min=40, nt_max=3000, t_min=5.0, t_max=80.0)
    slack = 3 + 5 * np.arange(b.n)  # gaps of uneven length after every curve's bins
    P_off = np.zeros(b.n + 1, np.int64)
    P_off[1:] = np.cumsum(b.nf + slack)
    return b, P_off


def _slack_intact(P_int, b, P_off, n_real):
    stride = int(P_off[-1])
    for r in range(n_real):
        for c in range(b.n):
            lo = r * stride + int(P_off[c]) + int(b.nf[c])
            hi = r * stride + int(P_off[c + 1])
            if not np.all(P_int[lo:hi] == CANARY):
                return False
    return True


@pytest.mark.parametrize("n_real,rhs", [(1, 0), (3, 0), (13, 0), (19, 4), (35, 0)])
def test_batch_writes_only_its_bins(lsp, n_real, rhs):
    """Noise batch: single realization, groups with their own CC/CS (3 in
    groups of 2; 13 in the automatic groups of 8, the last partial), and
    groups reading the window pass (19 at R = 4 and 35 in the automatic
    groups of 8, each with a partial last group)."""
    b, P_off = _batch_with_slack()
    n = n_real * int(P_off[-1])
    buf, P = _padded(n)
    mbuf, maxP = _padded(n_real * b.n)
    ctx = lsp.Context(0, batch_rhs=rhs)
    ctx.batch(_dev(b.t_off), _dev(b.t), _dev(b.f0), _dev(b.df), _dev(b.nf), seed=5, n_real=n_real,
              P_out=P, P_off=_dev(P_off), maxP=maxP, argmax=torch.empty(n_real * b.n, dtype=torch.int32,
                                                                          device="cuda"))
    ctx.sync(60.0)
    assert _pads_intact(buf, n) and _pads_intact(mbuf, n_real * b.n)
    P_int = buf.cpu().numpy()[PAD:PAD + n]
    assert _slack_intact(P_int, b, P_off, n_real)
    ctx.close()


@pytest.mark.parametrize("n_real", [1, 13])
def test_batch_host_output_keeps_its_slack(lsp, n_real):
    """A host P_out is staged through device memory; the slack its layout
    leaves between curves must come back as the caller left it."""
    b, P_off = _batch_with_slack(n_curves=7, seed=23)
    n = n_real * int(P_off[-1])
    buf = np.full(n + 2 * PAD, CANARY, dtype=np.int32)
    P = buf.view(np.float32)[PAD:PAD + n]
    ctx = lsp.Context(0)
    ctx.batch(b.t_off, b.t, b.f0, b.df, b.nf, seed=5, n_real=n_real, P_out=P, P_off=P_off,
              maxP=np.empty(n_real * b.n, np.float32), argmax=np.empty(n_real * b.n, np.int32))
    assert np.all(buf[:PAD] == CANARY) and np.all(buf[PAD + n:] == CANARY)
    assert _slack_intact(buf[PAD:PAD + n], b, P_off, n_real)
    ctx.close()


def test_floating_mean_batch_host_output_keeps_its_slack(lsp):
    b, P_off = _batch_with_slack(n_curves=7, seed=24)
    rng = np.random.default_rng(24)
    X = rng.normal(size=b.t.size)
    dy = rng.uniform(0.5, 2.0, b.t.size)
    n = int(P_off[-1])
    buf = np.full(n + 2 * PAD, CANARY, dtype=np.int32)
    P = buf.view(np.float32)[PAD:PAD + n]
    ctx = lsp.Context(0)
    ctx.batch_gls(b.t_off, b.t, X, b.f0, b.df, b.nf, dy=dy, P_out=P, P_off=P_off,
                  maxP=np.empty(b.n, np.float32), argmax=np.empty(b.n, np.int32))
    assert np.all(buf[:PAD] == CANARY) and np.all(buf[PAD + n:] == CANARY)
    assert _slack_intact(buf[PAD:PAD + n], b, P_off, 1)
    ctx.close()


def test_floating_mean_batch_writes_only_its_bins(lsp):
    b, P_off = _batch_with_slack(seed=22)
    rng = np.random.default_rng(4)
    X = rng.normal(size=b.t.size)
    dy = np.exp(rng.uniform(np.log(0.3), np.log(2.0), b.t.size))
    n = int(P_off[-1])
    buf, P = _padded(n)
    ctx = lsp.Context(0)
    ctx.batch_gls(_dev(b.t_off), _dev(b.t), _dev(X), _dev(b.f0), _dev(b.df), _dev(b.nf), dy=_dev(dy),
                  P_out=P, P_off=_dev(P_off), maxP=torch.empty(b.n, device="cuda"),
                  argmax=torch.empty(b.n, dtype=torch.int32, device="cuda"))
    ctx.sync(60.0)
    assert _pads_intact(buf, n)
    assert _slack_intact(buf.cpu().numpy()[PAD:PAD + n], b, P_off, 1)
    ctx.close()
