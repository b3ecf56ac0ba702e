"""The batch autotuner (lsp_autotune_batch) and the tuning table's JSON file.

A tuned batch must use the chosen launch shape and stay within oracle
parity; the table must survive a save / load round trip into a fresh
context, and a file written for another GPU must not be applied.
"""
import json
import os

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


def _batch(n=48, seed=515):
    from paper_1007_1658_gb300 import synth
    b = synth.noise_batch(n_curves=n, seed=seed, nt_min=200, nt_max=3000, t_min=30.0, t_max=300.0)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return b, (d(b.t_off), d(b.t), d(b.f0), d(b.df), d(b.nf))


def _batch_entries(path):
    with open(path) as fh:
        doc = json.load(fh)
    return doc, [e for e in doc["entries"] if e["kind"] == 2]


@pytest.mark.parametrize("n_real", [1, 8, 30])
def test_tuned_batch_uses_its_shape_and_matches_the_oracle(lsp, tmp_path, n_real):
    b, args = _batch()
    ctx = lsp.Context(0)
    chosen = ctx.autotune_batch(*args, n_real=n_real)
    path = tmp_path / "tune.json"
    ctx.tune_save(path)
    doc, entries = _batch_entries(path)
    assert len(entries) == 1
    e = entries[0]
    assert chosen["freqs_per_thread"] == e["F"] and chosen["batch_rhs"] == e["R"]
    # internal kernel mode -> public sin/cos mode: recurrence, three-term, packed three-term
    assert chosen["sincos_mode"] == {2: 2, 4: 3, 5: 4}[e["mode"]]
    seed = 4321
    maxP, argmax = ctx.batch(*args, seed=seed, n_real=n_real)
    ctx.sync(120.0)
    assert ctx.test_last_batch_shape() == (e["mode"], e["F"], e["R"], e["tailF"], e["tile"])
    maxP = maxP.cpu().numpy().reshape(n_real, b.n)
    for c in (0, 7, b.n - 1):
        for r in sorted({0, n_real - 1}):
            t = b.curve_t(c)
            X = oracle.noise(seed, c, r, t.size)
            ref = oracle.periodogram(t, X, b.f0[c], b.df[c], b.nf[c])
            assert abs(maxP[r, c] - ref.max()) <= 1e-4 * ref.max(), (c, r)
    # a fresh context takes the shape from the file
    ctx2 = lsp.Context(0)
    assert ctx2.tune_load(path) == len(doc["entries"])
    ctx2.batch(*args, seed=seed, n_real=n_real)
    ctx2.sync(120.0)
    assert ctx2.test_last_batch_shape() == (e["mode"], e["F"], e["R"], e["tailF"], e["tile"])
    ctx.close()
    ctx2.close()


def test_tuned_shapes_agree_with_the_default_and_the_oracle(lsp):
    """Every single-realization shape the tuner may pick, in the packed
    (internal mode 5) and scalar (4) three-term forms, gives the oracle's
    periodogram (full P of a few curves) and the same maxima as the first."""
    b, args = _batch(n=24, seed=616)
    P_off = np.zeros(b.n + 1, np.int64)
    P_off[1:] = np.cumsum(b.nf)
    P_off_d = torch.from_numpy(P_off).cuda()
    X = np.concatenate([oracle.noise(9, c, 0, int(b.t_off[c + 1] - b.t_off[c])) for c in range(b.n)])
    X_d = torch.from_numpy(X).cuda()
    refs = {c: oracle.periodogram(b.curve_t(c), X[b.t_off[c]:b.t_off[c + 1]], b.f0[c], b.df[c], b.nf[c])
            for c in (0, 11, b.n - 1)}
    base = None
    path_dir = os.environ.get("TMPDIR", "/tmp")
    for mode, F, tail, tile in [(m, F, tail, tile) for m in (5, 4) for F in (24, 16) for tail in (8, 4, 0)
                                for tile in (256, 128, 512)]:
        ctx = lsp.Context(0)
        # write a one-entry tuning file for this bucket, then load it
        ctx.autotune_batch(*args, n_real=1)
        path = os.path.join(path_dir, "lsp_tune_%d_%d_%d_%d_%d.json" % (os.getpid(), mode, F, tail, tile))
        ctx.tune_save(path)
        doc, entries = _batch_entries(path)
        entries[0].update(mode=mode, F=F, R=1, tailF=tail, tile=tile)
        with open(path, "w") as fh:
            fh.write('{"lsp_tune": 1, "device": "%s", "entries": [\n' % doc["device"])
            fh.write(json.dumps(entries[0]) + "\n]}\n")
        ctx2 = lsp.Context(0)
        assert ctx2.tune_load(path) == 1
        os.remove(path)
        P = torch.empty(int(P_off[-1]), dtype=torch.float32, device="cuda")
        maxP, _ = ctx2.batch(args[0], args[1], args[2], args[3], args[4], X=X_d, P_out=P, P_off=P_off_d,
                             maxP=torch.empty(b.n, dtype=torch.float32, device="cuda"),
                             argmax=torch.empty(b.n, dtype=torch.int32, device="cuda"))
        ctx2.sync(120.0)
        assert ctx2.test_last_batch_shape() == (mode, F, 1, tail, tile)
        Pn = P.cpu().numpy()
        for c, ref in refs.items():
            assert_parity(Pn[P_off[c]:P_off[c] + b.nf[c]], ref, what="mode %d F %d tail %d tile %d curve %d"
                          % (mode, F, tail, tile, c))
        m = maxP.cpu().numpy().astype(np.float64)
        if base is None:
            base = m
        assert np.max(np.abs(m - base) / base) <= 2e-5
        ctx.close()
        ctx2.close()


def test_tuning_file_of_another_gpu_is_not_applied(lsp, tmp_path):
    b, args = _batch(n=8, seed=717)
    ctx = lsp.Context(0)
    ctx.autotune_batch(*args, n_real=1)
    path = tmp_path / "tune.json"
    ctx.tune_save(path)
    txt = path.read_text()
    doc = json.loads(txt)
    other = tmp_path / "other.json"
    other.write_text(txt.replace('"device": "%s"' % doc["device"], '"device": "some other GPU"'))
    ctx2 = lsp.Context(0)
    assert ctx2.tune_load(other) == 0
    bad = tmp_path / "bad.json"
    bad.write_text("not a tuning file\n")
    with pytest.raises(lsp.LspError) as e:
        ctx2.tune_load(bad)
    assert e.value.status == lsp.ERR_INVALID_ARG
    ctx.close()
    ctx2.close()


def test_single_curve_tuning_round_trip(lsp, tmp_path):
    """lsp_autotune's entry survives lsp_tune_save / lsp_tune_load, and a fresh
    context that loaded it still matches the oracle on a curve of that bucket."""
    from paper_1007_1658_gb300 import synth
    c = synth.plain_1k()
    ctx = lsp.Context(0)
    chosen = ctx.autotune(c.t.size, c.nf)
    path = tmp_path / "tune1.json"
    ctx.tune_save(path)
    doc, _ = _batch_entries(path)
    single = [e for e in doc["entries"] if e["kind"] == 1]
    assert len(single) == 1
    e = single[0]
    assert (e["sincos"], e["F"]) == (chosen["sincos_mode"], chosen["freqs_per_thread"])
    ctx2 = lsp.Context(0)
    assert ctx2.tune_load(path) == 1
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    P = ctx2.periodogram(d(c.t), d(c.X), c.f0, c.df, c.nf)
    ctx2.sync(60.0)
    assert_parity(P.cpu().numpy(), oracle.periodogram(c.t, c.X, c.f0, c.df, c.nf), what="loaded tuning entry")
    ctx.close()
    ctx2.close()


def test_tuned_multi_realization_shapes_match_the_oracle(lsp):
    """Multi-realization shapes the tuner may pick, including the tiles of 256
    and 512, every group size and the packed strips (internal mode 5), with 24
    realizations (four groups or more at R = 2 and 4, so CC and CS come from
    the window pass; at R = 8 the three groups keep their own): each agrees
    with the oracle on the maxima of a few (curve, realization) pairs, and
    with the others."""
    b, args = _batch(n=24, seed=717)
    n_real, seed = 24, 2718
    refs = {}
    for c in (0, 9, b.n - 1):
        for r in (0, 13, n_real - 1):
            t = b.curve_t(c)
            refs[c, r] = oracle.periodogram(t, oracle.noise(seed, c, r, t.size), b.f0[c], b.df[c], b.nf[c]).max()
    base = None
    path_dir = os.environ.get("TMPDIR", "/tmp")
    for mode, F, R, tile in ((4, 12, 4, 128), (4, 12, 4, 256), (4, 8, 4, 512), (4, 8, 8, 128), (4, 16, 2, 128),
                             (5, 12, 4, 128), (5, 8, 8, 128), (5, 16, 2, 128)):
        ctx = lsp.Context(0)
        ctx.autotune_batch(*args, n_real=n_real)
        path = os.path.join(path_dir, "lsp_tune_mr_%d_%d_%d_%d.json" % (os.getpid(), F, R, tile))
        ctx.tune_save(path)
        doc, entries = _batch_entries(path)
        entries[0].update(mode=mode, F=F, R=R, tailF=0, tile=tile)
        with open(path, "w") as fh:
            fh.write('{"lsp_tune": 1, "device": "%s", "entries": [\n' % doc["device"])
            fh.write(json.dumps(entries[0]) + "\n]}\n")
        ctx2 = lsp.Context(0)
        assert ctx2.tune_load(path) == 1
        os.remove(path)
        maxP, _ = ctx2.batch(*args, seed=seed, n_real=n_real)
        ctx2.sync(120.0)
        assert ctx2.test_last_batch_shape() == (mode, F, R, 0, tile)
        m = maxP.cpu().numpy().astype(np.float64).reshape(n_real, b.n)
        for (c, r), ref in refs.items():
            assert abs(m[r, c] - ref) <= 1e-4 * ref, (mode, F, R, tile, c, r)
        if base is None:
            base = m
        assert np.max(np.abs(m - base) / base) <= 2e-5, (mode, F, R, tile)
        ctx.close()
        ctx2.close()
