"""GPU parity of the reverse-mode adjoint (d fitness / d ERC) against the FP64
oracle's reverse-mode gradient, plus the autograd wrapper and the Adam
kernel.  Trials whose fitness is excluded as ill-conditioned or ambiguous,
whose FP32 evaluation overflows at an intermediate node, or whose FP64
gradient is not finite, are skipped and counted."""
import numpy as np
import pytest
import torch

import synth
import parity as PA

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_30954_gb300 as pkg
    pkg.lib()
    return pkg


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def grad_case(gg, w, mode="smse", sample=None, name=None):
    """Adjoint of every (or every sampled) trial against the oracle; the
    counts go to the parity report, with the gradient entries that pass
    only through the FP32 floor term of the tolerance."""
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    op, cv = dev(w["op"]), dev(w["cval"])
    hs = dev(w["heights"]) if len(set(w["heights"].tolist())) > 1 else None
    flags = (gg.F_GRAD_MSE if mode == "mse" else 0) | (gg.F_POW if w.get("uses_pow") else 0)
    smse, dc = ds.grad_batch(op, cv, hs, flags=flags)
    ds.sync()
    smse, dc = smse.cpu().numpy(), dc.cpu().numpy()
    ds.close()
    idx = list(range(w["P"])) if sample is None else list(sample)
    tally, fit_tally, n_floor, n_ill = PA.check_gradients(w, idx, dc, smse, mode)
    if name:
        PA.report(f"{name} (floor-only {n_floor}, ill-cond. {n_ill})", "grads", tally)
    return tally, fit_tally


@pytest.mark.parametrize("mode", ["smse", "mse"])
def test_adjoint_small_c4(gg, mode):
    w = PA.build("c4", 2500, 48)
    t, tf = grad_case(gg, w, mode, name=f"adjoint {mode} c4 2,500 rows")
    assert t.failed == 0 and tf.failed == 0, (repr(t), repr(tf))
    assert t.checked >= 24, repr(t)


@pytest.mark.parametrize("cfg,n_rows,n_trials", [("c2", 3000, 40), ("c3", 2100, 32),
                                                  ("c1", 1000, 64), ("t2", 3000, 48)])
def test_adjoint_other_shapes(gg, cfg, n_rows, n_trials):
    w = PA.build(cfg, n_rows, n_trials)
    t, tf = grad_case(gg, w, name=f"adjoint {cfg} {n_rows} rows")
    assert t.failed == 0 and tf.failed == 0, (repr(t), repr(tf))
    assert t.checked >= n_trials // 3, repr(t)


@pytest.mark.parametrize("cfg,n_sample", [("c4", 128), ("c5", 16)])
def test_adjoint_full_size_sampled(gg, cfg, n_sample):
    """The gradient workload (1,024 x h5 over 50,000 rows) and the largest
    one (16,384 x h6 over 1,000,000 rows, where the adjoint recomputes node
    values row block by row block): sampled trials against the oracle."""
    w = PA.build(cfg)
    sample = np.random.default_rng(3).choice(w["P"], n_sample, replace=False).tolist()
    t, tf = grad_case(gg, w, sample=sample, name=f"adjoint full-size {w['name']}")
    assert t.failed == 0 and tf.failed == 0, (repr(t), repr(tf))
    assert t.checked >= n_sample // 2, repr(t)


def test_autograd_function_and_adam(gg):
    w = PA.build("c4", 3000, 32)
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    op = dev(w["op"])
    cv = dev(w["cval"]).requires_grad_(True)
    smse = gg.ScaledMSE.apply(cv, op, ds)
    smse_ref, dc_ref = ds.grad_batch(op, cv.detach().clone())
    fin = torch.isfinite(smse)
    (smse[fin] * 2.0).sum().backward()
    torch.cuda.synchronize()
    assert torch.equal(smse, smse_ref)
    g = cv.grad.clone()
    assert torch.allclose(g[fin], 2.0 * dc_ref[fin])
    # Adam kernel vs the textbook update on the same gradient
    c = dev(w["cval"])
    m = torch.zeros_like(c)
    v = torch.zeros_like(c)
    cn, mn, vn = (x.cpu().numpy().astype(np.float64) for x in (c, m, v))
    gn = dc_ref.cpu().numpy().astype(np.float64)
    erc = w["op"] == synth.ERC
    for t in (1, 2, 3):
        gg.adam_step(op, c, dc_ref, m, v, t, lr=0.05)
        mn = np.where(erc, 0.9 * mn + 0.1 * gn, mn)
        vn = np.where(erc, 0.999 * vn + 0.001 * gn * gn, vn)
        step = 0.05 * (mn / (1 - 0.9 ** t)) / (np.sqrt(vn / (1 - 0.999 ** t)) + 1e-8)
        cn = np.where(erc, cn - step, cn)
    torch.cuda.synchronize()
    np.testing.assert_allclose(c.cpu().numpy(), cn, rtol=1e-5, atol=1e-6)
    ds.close()


def test_constant_tuning_reduces_fitness(gg):
    w = PA.build("c4", 5000, 64)
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    op = dev(w["op"])
    c = dev(w["cval"])
    m, v = torch.zeros_like(c), torch.zeros_like(c)
    s0 = ds.eval_batch(op, c)[0].clone()
    for t in range(1, 21):
        _, g = ds.grad_batch(op, c)
        g = torch.nan_to_num(g, nan=0.0, posinf=0.0, neginf=0.0)
        gg.adam_step(op, c, g, m, v, t, lr=0.05)
    s1 = ds.eval_batch(op, c)[0]
    ds.sync()
    fin = torch.isfinite(s0) & torch.isfinite(s1)
    improved = (s1[fin] <= s0[fin] * (1 + 1e-6)).float().mean().item()
    assert improved >= 0.8, improved
    assert (s1[fin] < s0[fin] * 0.999).sum().item() >= 4
    ds.close()


def test_adjoint_deep_stack_many_ercs(gg):
    """Full height-6 trees (every leaf active; internal nodes +, -, AQ, x)
    whose 64 leaves are 48 ERCs and 16 features: programs of 64
    instructions that need the deepest forward stack (5 slots) and carry 48
    ERCs (two rounds of the per-pass ERC reduction).  In the staged adjoint
    the forward stack and the ERC partials share their shared-memory bytes;
    here both are at their largest."""
    import synth
    w = PA.build("c5", 3000, 32)
    rng = np.random.default_rng(11)
    P, S = w["op"].shape
    n_int = S // 2  # heap positions 0 .. 62 are internal, 63 .. 126 leaves
    op = np.empty_like(w["op"])
    cv = np.zeros_like(w["cval"])
    op[:, :n_int] = rng.choice([synth.ADD, synth.SUB, synth.AQ, synth.MUL], size=(P, n_int),
                               p=[0.35, 0.35, 0.2, 0.1])
    leaves = np.full((P, S - n_int), synth.ERC, dtype=op.dtype)
    for p in range(P):
        k = rng.choice(S - n_int, 16, replace=False)
        leaves[p, k] = synth.FEAT0 + rng.integers(0, w["F"], 16)
    op[:, n_int:] = leaves
    cv[:, n_int:] = rng.uniform(-1, 1, (P, S - n_int)).astype(cv.dtype)
    w["op"], w["cval"] = op, cv
    assert all(int(np.sum(op[p] == synth.ERC)) == 48 for p in range(P))
    t, tf = grad_case(gg, w, name="adjoint full h6 trees, 48 ERCs each")
    assert t.failed == 0 and tf.failed == 0, (repr(t), repr(tf))
    assert t.checked >= P // 2, repr(t)
