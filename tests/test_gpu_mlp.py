"""The learned initial-state proposal: tensor-core forward/backward against
the FP64 oracle's MLP (weights and inputs from a seeded generator, rounded
to bf16 as the kernels see them), training progress, checkpoint resume and
corruption, and what the trained network gains over plain LM."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2608_07580_b300 import firert
    return torch, firert


def _bf16(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def test_gradients_match_oracle(env):
    torch, fr = env
    t = synth.make_tables()
    ctx = fr.Context(t)
    H = 64
    mlp = fr.MLP(ctx, hidden=H, seed=1)
    D = mlp.din
    rng = np.random.default_rng(4)
    p = {"W1": rng.normal(0, 0.08, (H, D)), "b1": rng.normal(0, 0.1, H),
         "W2": rng.normal(0, 0.15, (H, H)), "b2": rng.normal(0, 0.1, H),
         "W3": rng.normal(0, 0.15, (16, H)), "b3": rng.normal(0, 0.1, 16),
         "mean": np.zeros(D), "istd": np.ones(D)}
    mlp.params(p)
    ref = {k: _bf16(p[k]) if k.startswith("W") else p[k] for k in ("W1", "b1", "W2", "b2", "W3", "b3")}
    # The kernels store h1 and h2 (the next layer's tensor-core operand) in
    # bf16, which moves a pre-activation by up to ~2^-8 of the norm of its
    # terms; a unit that close to 0 may take the other side of its ReLU gate
    # than in FP64, a discrete change no rounding bound covers. The batch is
    # therefore drawn from candidates whose pre-activations (FP64, through
    # the bf16 weights and inputs) all lie farther than 2^-7 of that norm
    # from zero, and the oracle is the unmodified FP64 backward.
    cand = rng.normal(size=(1024, D))
    cand[:, 284:] = 0
    xc = _bf16(cand)
    a1, a2, _ = oracle.mlp_forward(ref, xc)
    n1 = np.sqrt((xc ** 2) @ (ref["W1"] ** 2).T)
    h1 = np.maximum(a1, 0.0)
    n2 = np.sqrt((h1 ** 2) @ (ref["W2"] ** 2).T)
    clear = np.all(np.abs(a1) > 2 ** -7 * n1, axis=1) & np.all(np.abs(a2) > 2 ** -7 * n2, axis=1)
    keep = np.flatnonzero(clear)
    B = (min(keep.size, 256) // 8) * 8
    assert B >= 64, keep.size
    x = cand[keep[:B]].astype(np.float32)
    tgt = np.tanh(rng.normal(size=(B, 16))).astype(np.float32)
    msk = (rng.uniform(size=(B, 16)) < 0.8).astype(np.float32)
    msk[:, 9:] = 0
    g, loss = mlp.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda(),
                            torch.from_numpy(msk).cuda())
    lo, go, _ = oracle.mlp_backward(ref, _bf16(x), tgt, msk, n_out=9)
    assert abs(loss / lo - 1) < 2e-2
    bound = {"W1": 2e-2, "b1": 2e-2, "W2": 2e-2, "b2": 2e-2, "W3": 2e-2, "b3": 2e-2}
    pairs = (("W1", g["W1"], go["W1"]), ("b1", g["b1"], go["b1"]), ("W2", g["W2"], go["W2"]),
             ("b2", g["b2"], go["b2"]), ("W3", g["W3T"].T, go["W3"]), ("b3", g["b3"], go["b3"]))
    for name, a, b in pairs:
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = float(np.sum(a * b) / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert rel < bound[name] and cos > 0.998, (name, rel, cos)


def test_training_reduces_loss_and_resumes(env, tmp_path):
    torch, fr = env
    t = synth.make_tables()
    ctx = fr.Context(t)
    mlp = fr.MLP(ctx, hidden=256, seed=2)
    l0 = mlp.train(60, batch=2048, lr=2e-3, seed=5)
    assert np.all(np.isfinite(l0))
    assert l0[-10:].mean() < 0.6 * l0[:5].mean()
    ck = tmp_path / "mlp.ckpt"
    mlp.save(ck)
    la = mlp.train(8, batch=2048, lr=2e-3, seed=5)
    mlp2 = fr.MLP(ctx, hidden=256, seed=99)
    mlp2.load(ck)
    lb = mlp2.train(8, batch=2048, lr=2e-3, seed=5)
    assert np.allclose(la, lb, rtol=1e-4, atol=1e-8)
    raw = bytearray(ck.read_bytes())
    raw[200] ^= 0xFF
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(raw))
    with pytest.raises(fr.FireError):
        mlp2.load(bad)


def test_learned_start_gains_over_plain_lm(env):
    """A trained network cuts the stage-1 LM iterations of the fire pixels
    (where a proposal carries information; the non-fire pixels start at
    alpha = 0 in plain LM, which is already close); plain LM judges it: the
    learned-start retrieval against the oracle's default-start fit at the
    full bar."""
    torch, fr = env
    import sys
    sys.path.insert(0, __import__("os").path.dirname(__file__))
    from scenes import config1
    t, tr, L = config1(seed=3)
    ctx = fr.Context(t)
    mlp = fr.MLP(ctx, hidden=512, seed=3)
    mlp.train(3000, batch=4096, lr=1e-3, seed=11)
    ctx.set_mlp(mlp)
    Ld = torch.from_numpy(L).cuda()
    wd = torch.from_numpy(tr.wv_bin.astype(np.int16)).cuda()
    plain = {k: v.cpu().numpy() for k, v in ctx.retrieve(Ld, wd).items()}
    learned = {k: v.cpu().numpy() for k, v in ctx.retrieve(Ld, wd, learned_start=True).items()}
    it_p = plain["iters"].astype(np.int64).sum(1).mean()
    it_l = learned["iters"].astype(np.int64).sum(1).mean()
    f = tr.kind == 1
    f1_p = plain["iters"][f, 0].astype(np.int64).mean()
    f1_l = learned["iters"][f, 0].astype(np.int64).mean()
    print("mean iterations plain %.2f learned %.2f; fire pixels' stage 1 plain %.2f learned %.2f; fallback %.3f"
          % (it_p, it_l, f1_p, f1_l, np.mean((learned["status"] & 32) > 0)))
    assert f1_l < f1_p
    # plain LM judges the learned start: the learned-start retrieval against
    # the oracle's default-start fit, at the full bar
    from scenes import parity_stats, summary
    o = oracle.retrieve(t, L, tr.wv_bin)
    s = parity_stats(o, learned)
    print("learned start vs oracle:", summary(s))
    assert s["pool"] >= 100
    assert s["rate"] >= 0.999, summary(s)
    # accuracy against the seeded truth, plain and learned start
    fire = np.flatnonzero((tr.kind == 1) & ((o["status"] & 23) == 0))
    T = tr.single[fire, 1]
    for name, r in (("plain", plain), ("learned", learned)):
        e = r["ET"][fire] - T
        print(f"{name}: E[T] vs truth RMSE {np.sqrt(np.mean(e ** 2)):.2f} K, MAE {np.mean(np.abs(e)):.2f} K")
