"""GPU parity of the false-alarm surrogate: features, forward, gradients, Adam,
checkpoints -- each against the FP64 numpy oracle (oracle/surrogate.py).

Tolerances: features 0..15 to 1e-5 (relative or absolute), window heights to
2e-5 absolute (FP32 window sums against FP64), their frequencies exactly where
the heights are not near-ties; network quantiles to 1e-4 relative and
gradients to 1e-3 relative (per tensor, in norm) with FP32 activations, 5e-2
with BF16 activations (8-bit mantissas through three layers and the head's exp).
"""
import numpy as np
import pytest

import oracle
from oracle import surrogate as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lsp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_1658_gb300 import build, lsp as L
    build.build()
    return L


@pytest.fixture()
def ctx(lsp):
    c = lsp.Context(0)
    yield c
    c.close()


def _patterns(n=12, seed=21, lo=200, hi=3000):
    from paper_1007_1658_gb300 import synth
    return synth.noise_batch(n_curves=n, seed=seed, nt_min=lo, nt_max=hi, t_min=20.0, t_max=400.0)


def _check_features(got, ref):
    assert np.allclose(got[:16], ref[:16], rtol=1e-5, atol=1e-5), np.c_[got[:16], ref[:16]]
    assert np.allclose(got[16:24], ref[16:24], atol=2e-5)
    h = ref[16:24]
    for r in range(8):
        near = (r > 0 and abs(h[r] - h[r - 1]) < 1e-4) or (r < 7 and abs(h[r] - h[r + 1]) < 1e-4)
        if not near:
            assert abs(got[24 + r] - ref[24 + r]) <= 1e-6 * max(1.0, abs(ref[24 + r])), r


def test_features_match_oracle(ctx):
    b = _patterns()
    got = ctx.fap_features(b.t_off, b.t, b.f0, b.df, b.nf)
    for c in range(b.n):
        ref = S.features(b.curve_t(c), b.f0[c], b.df[c], b.nf[c])
        _check_features(got[c].astype(np.float64), ref)
    # device arrays give the same bits
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gd = ctx.fap_features(d(b.t_off), d(b.t), d(b.f0), d(b.df), d(b.nf))
    ctx.sync(30.0)
    assert np.array_equal(gd.cpu().numpy(), got)


def _long_patterns():
    """Patterns on both sides of the shared-memory sort's 32,768 gaps, longer
    random ones with exponential gaps (neighbouring order statistics well
    apart, so a rank off by one shows), and the paper-shape cadence."""
    from paper_1007_1658_gb300 import synth
    rng = np.random.default_rng(5150)
    ts = [np.sort(rng.uniform(0.0, 300.0, 32_769)), np.sort(rng.uniform(0.0, 300.0, 32_770)),
          np.cumsum(rng.exponential(0.01, 60_001)), np.cumsum(rng.exponential(0.02, 120_000))]
    ts.append(synth.corot_382k().t)
    return ts


def test_features_of_long_patterns_match_oracle(ctx):
    """Patterns of more than 32,769 samples take the radix select of the five
    cadence order statistics instead of the shared-memory sort; both paths
    against the oracle, and the quantile features against the FP32 gaps'
    exact order statistics (to one float ulp of the log)."""
    ts = _long_patterns()
    off = np.concatenate([[0], np.cumsum([t.size for t in ts])]).astype(np.int64)
    nf = np.array([1500] * len(ts), np.int64)  # a short window grid keeps the oracle quick
    df = np.array([1.0 / (4.0 * (t[-1] - t[0])) for t in ts])
    got = ctx.fap_features(off, np.concatenate(ts), df.copy(), df, nf)
    for c, t in enumerate(ts):
        ref = S.features(t, df[c], df[c], nf[c])
        _check_features(got[c].astype(np.float64), ref)
        g32 = np.sort(np.diff(t).astype(np.float32))
        M, T = g32.size, t[-1] - t[0]
        for i, p in enumerate((0.05, 0.25, 0.5, 0.75, 0.95)):
            q = float(g32[int(np.floor(p * (M - 1)))])
            want = np.float32(np.log(max(q, 1e-12 * T) / (T / M)))
            assert abs(got[c, 6 + i] - want) <= 1.2e-7 * max(1.0, abs(want)), (c, p, got[c, 6 + i], want)


def test_features_even_grid_and_unsorted(ctx, lsp):
    N, dt = 400, 0.25
    t = np.arange(N) * dt
    T = (N - 1) * dt
    df = 1.0 / (4 * T)
    f = ctx.fap_features(np.array([0, N], np.int64), t, np.array([df]), np.array([df]), np.array([2 * N], np.int64))[0]
    ref = S.features(t, df, df, 2 * N)
    _check_features(f.astype(np.float64), ref)
    assert np.allclose(f[6:11], 0.0, atol=1e-6)
    bad = t.copy()
    bad[[10, 11]] = bad[[11, 10]]
    with pytest.raises(lsp.LspError) as e:
        ctx.fap_features(np.array([0, N], np.int64), bad, np.array([df]), np.array([df]), np.array([2 * N], np.int64))
        ctx.sync(10.0)
    assert e.value.status == lsp.ERR_NONFINITE
    # the same on the radix-select path (more than 32,769 samples)
    N2 = 40_000
    bad2 = np.arange(N2) * dt
    bad2[[30_000, 30_001]] = bad2[[30_001, 30_000]]
    df2 = 1.0 / (4 * (N2 - 1) * dt)
    with pytest.raises(lsp.LspError) as e:
        ctx.fap_features(np.array([0, N2], np.int64), bad2, np.array([df2]), np.array([df2]),
                         np.array([500], np.int64))
        ctx.sync(10.0)
    assert e.value.status == lsp.ERR_NONFINITE


def _random_model(hidden, seed):
    rng = np.random.default_rng(seed)
    ps = [p + 0.05 * rng.normal(size=p.shape) for p in S.init_params(rng, hidden=hidden)]
    mu = rng.normal(size=32) * 0.1
    sig = np.exp(rng.normal(size=32) * 0.2)
    flat = np.concatenate([p.reshape(-1) for p in ps] + [mu, sig]).astype(np.float32)
    ps32 = [p.astype(np.float32).astype(np.float64) for p in ps]
    return flat, ps32, mu.astype(np.float32).astype(np.float64), sig.astype(np.float32).astype(np.float64)


def _rows(B, seed):
    rng = np.random.default_rng(seed)
    feat = rng.normal(size=(B, 32)).astype(np.float32)
    counts = np.column_stack([rng.integers(200, 20000, B), rng.integers(400, 40000, B)]).astype(np.float32)
    base = S.eq3_quantile(counts[:, :1].astype(np.float64), counts[:, 1:].astype(np.float64), S.LEVELS[None, :])
    y = (base[:, 4] * np.exp(rng.normal(0, 0.2, B))).astype(np.float32)
    return feat, counts, y


@pytest.mark.parametrize("fp32,tol", [(1, 1e-3), (0, 5e-2)])
def test_forward_and_gradients_match_oracle(lsp, fp32, tol):
    H, B = 64, 300
    ctx = lsp.Context(0, mlp_fp32=fp32)
    flat, ps, mu, sig = _random_model(H, 3)
    ctx.fap_set_params(flat, hidden=H)
    feat, counts, y = _rows(B, 4)
    X = (feat.astype(np.float64) - mu) / sig
    q_ref, loss_ref, cache = S.mlp_forward(ps, X, counts.astype(np.float64), y.astype(np.float64))
    g_ref = S.mlp_backward(ps, cache, y.astype(np.float64))
    q = ctx.fap_eval(feat, counts)
    # BF16 activations (8-bit mantissa) through three layers and the exp of the head
    assert np.max(np.abs(q - q_ref) / q_ref) <= (1e-4 if fp32 else 5e-2)
    g, loss = ctx.fap_gradients(feat, counts, y)
    assert abs(loss - loss_ref) <= tol * abs(loss_ref)
    o = 0
    for gr in g_ref:
        n = gr.size
        got = g[o:o + n].astype(np.float64)
        o += n
        assert np.linalg.norm(got - gr.reshape(-1)) <= tol * np.linalg.norm(gr) + 1e-12
    ctx.close()


def test_adam_step_matches_oracle(lsp):
    H, B = 32, 256
    ctx = lsp.Context(0, mlp_fp32=1)
    flat, ps, mu, sig = _random_model(H, 5)
    ctx.fap_set_params(flat, hidden=H)
    feat, counts, y = _rows(B, 6)
    X = (feat.astype(np.float64) - mu) / sig
    _, _, cache = S.mlp_forward(ps, X, counts.astype(np.float64), y.astype(np.float64))
    g = S.mlp_backward(ps, cache, y.astype(np.float64))
    zeros = [np.zeros_like(p) for p in ps]
    new, _, _ = S.adam_step(ps, g, zeros, zeros, step=1, lr=1e-3)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rows = d(np.arange(B, dtype=np.int32))
    ctx.fap_train_step(rows, d(feat), d(counts), d(y), 1e-3)
    got = ctx.fap_get_params()
    o = 0
    for p0, p1 in zip(ps, new):
        n = p0.size
        step_ref = (p1 - p0).reshape(-1)
        step_got = got[o:o + n].astype(np.float64) - p0.reshape(-1)
        o += n
        # the first Adam step is lr * sign(g) where |g| >> eps: compare the moves
        big = np.abs(step_ref) > 5e-4
        assert np.mean(np.abs(step_got[big] - step_ref[big]) <= 1e-5) > 0.99
    ctx.close()


def test_checkpoint_round_trip(lsp, tmp_path):
    ctx = lsp.Context(0)
    feat, counts, y = _rows(128, 7)
    ctx.fap_init(feat, hidden=16, seed=9)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for _ in range(3):
        ctx.fap_train_step(d(np.arange(128, dtype=np.int32)), d(feat), d(counts), d(y), 1e-3)
    path = tmp_path / "m.bin"
    ctx.fap_save(path)
    q0 = ctx.fap_eval(feat, counts)
    other = lsp.Context(0)
    other.fap_load(path)
    assert np.array_equal(other.fap_get_params(), ctx.fap_get_params())
    assert np.array_equal(other.fap_eval(feat, counts), q0)
    raw = bytearray(path.read_bytes())
    raw[100] ^= 0x40
    bad = tmp_path / "bad.bin"
    bad.write_bytes(bytes(raw))
    with pytest.raises(lsp.LspError):
        other.fap_load(bad)
    ctx.close()
    other.close()


def test_untrained_context_reports_no_model(lsp):
    ctx = lsp.Context(0)
    feat, counts, _ = _rows(4, 8)
    with pytest.raises(lsp.LspError) as e:
        ctx.fap_eval(feat, counts)
    assert e.value.status == lsp.ERR_NO_MODEL
    ctx.close()


def test_committed_model_beats_eq3_against_monte_carlo(lsp):
    """What the trained network gains over the method without it: on held-out
    patterns, its max-peak quantiles are closer to brute-force Monte Carlo than
    Eq. 3's (exponent N_f), and within 5% at every level."""
    from paper_1007_1658_gb300 import surrogate as SU
    ctx = lsp.Context(0)
    ctx.fap_load(SU.DEFAULT_MODEL)
    jd = SU.evaluate(ctx, n_patterns=48, n_real=3000, seed=424242)
    sur = np.array(jd["mean_rel_err_surrogate"])
    eq3 = np.array(jd["mean_rel_err_eq3"])
    assert sur.max() <= 0.05, sur
    assert sur.max() < eq3.max() and sur.mean() < eq3.mean(), (sur, eq3)
    assert jd["gpu_s_ratio"] >= 100.0
    ctx.close()


def test_quick_training_improves_on_eq3(lsp):
    """Training from scratch on engine-generated noise periodograms lowers the
    validation pinball loss below Eq. 3's (the untrained network's)."""
    from paper_1007_1658_gb300 import surrogate as SU
    ctx = lsp.Context(0)
    tr = SU.train(ctx, n_patterns=2048, n_real=4, steps=150, batch=2048, lr=1e-3, warmup_steps=10, n_val=256,
                  eval_every=50, verbose=False)
    assert tr["val_loss_best"] < tr["val_loss_eq3"]
    ctx.close()


def _train_set(ctx, n_pat, n_real, seed):
    from paper_1007_1658_gb300 import surrogate as SU, synth
    b = synth.noise_batch(n_curves=n_pat, seed=seed, nt_min=200, nt_max=4000, t_min=30.0, t_max=500.0)
    pats = SU.DevicePatterns(b, torch.device("cuda", 0))
    y = SU.mc_maxima(ctx, pats, n_real, seed=seed + 17).contiguous()
    f = ctx.fap_features(pats.t_off, pats.t, pats.f0, pats.df, pats.nf)
    return b, pats, f, y


def test_lsp_fap_train_through_the_c_abi(lsp):
    """The whole loop in the library (lsp_fap_train, called through ctypes):
    its first validation loss is the pinball loss of Eq. 3's quantiles against
    the validation maxima (recomputed here from the FP64 oracle's Eq. 3), the
    kept weights end below it, the report agrees with the histories, and the
    same seed gives the same weights."""
    ctx = lsp.Context(0)
    b, pats, feats, y = _train_set(ctx, 768, 4, 9100)
    vb, vpats, vfeats, vy = _train_set(ctx, 96, 8, 9200)
    params = []
    reps = []
    for _ in range(2):
        ctx.fap_init(feats, hidden=64, seed=5)
        rep = ctx.fap_train(feats, pats.counts, y.reshape(-1).contiguous(), vfeats, vpats.counts, vy, steps=240,
                            batch=1024, lr=1e-3, warmup_steps=20, eval_every=40, seed=77)
        params.append(ctx.fap_get_params())
        reps.append(rep)
    rep = reps[0]
    assert np.array_equal(params[0], params[1]) and reps[0]["val_history"] == reps[1]["val_history"]
    # pass before training: the untrained head is Eq. 3
    n = np.diff(vb.t_off).astype(np.float64)
    q = S.eq3_quantile(n[:, None], vb.nf.astype(np.float64)[:, None], np.array(S.LEVELS)[None, :])
    yy = vy.cpu().numpy().astype(np.float64)  # [n_real][n_pat]
    u = yy[:, :, None] - q[None, :, :]
    lv = np.array(S.LEVELS)
    ref = np.mean(np.sum(np.maximum(lv * u, (lv - 1.0) * u), axis=2))
    assert abs(rep["val_loss_initial"] - ref) <= 1e-3 * ref, (rep["val_loss_initial"], ref)
    assert rep["evaluations"] == 2 + (240 - 1) // 40 == len(rep["val_history"])
    assert np.isnan(rep["train_history"][0]) and np.all(np.isfinite(rep["train_history"][1:]))
    assert rep["val_loss_best"] == min(rep["val_history"])
    assert rep["best_step"] in [0] + [min(240, 40 * (e + 1)) for e in range(rep["evaluations"] - 1)]
    assert rep["val_loss_best"] < rep["val_loss_initial"]
    # the context now holds the kept weights: evaluating them reproduces the best loss
    qv = ctx.fap_eval(vfeats, vpats.counts).cpu().numpy().astype(np.float64)
    u = yy[:, :, None] - qv[None, :, :]
    got = np.mean(np.sum(np.maximum(lv * u, (lv - 1.0) * u), axis=2))
    assert abs(got - rep["val_loss_best"]) <= 1e-4 * got
    ctx.close()


def test_lsp_fap_train_refuses_bad_schedules(lsp):
    ctx = lsp.Context(0)
    _, pats, feats, y = _train_set(ctx, 32, 2, 9300)
    ctx.fap_init(feats, hidden=16, seed=1)
    yy = y.reshape(-1).contiguous()
    for kw in (dict(steps=0), dict(batch=0), dict(lr=0.0), dict(lr_final=1.5), dict(warmup_steps=50, steps=10),
               dict(weight_decay=-1.0)):
        args = dict(steps=10, batch=64, lr=1e-3)
        args.update(kw)
        with pytest.raises(lsp.LspError) as e:
            ctx.fap_train(feats, pats.counts, yy, feats, pats.counts, y, **args)
        assert e.value.status == lsp.ERR_INVALID_ARG
    with pytest.raises(lsp.LspError) as e:  # host tables are refused
        ctx.fap_train(feats.cpu(), pats.counts, yy, feats, pats.counts, y, steps=10, batch=64)
    assert e.value.status == lsp.ERR_INVALID_ARG
    ctx.close()
