"""GPU parity of the device GOM step (donor copy, changed test, accept or
revert, masked evaluation) against the NumPy oracle of Algorithm 1:
bit-exact, since all of it is byte and index work."""
import numpy as np
import pytest
import torch

from oracle import gom
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


def fos_of(stride):
    """One subset per template node: the node and its two children."""
    return [[i] + [c for c in (2 * i + 1, 2 * i + 2) if c < stride] for i in range(stride)]


def test_fos_sweep_matches_oracle(gg):
    rng = np.random.default_rng(11)
    P, h, F = 300, 4, 6
    pop_op, pop_cv, _ = synth.random_templates(rng, P, h, h, synth.FULL_SET, F, 0.7)
    stride = pop_op.shape[1]
    fos = fos_of(stride)
    off = np.cumsum([0] + [len(s) for s in fos]).astype(np.int32)
    nodes = np.concatenate(fos).astype(np.int32)
    order = np.argsort(rng.random((P, stride)), axis=1)
    X = rng.uniform(-2, 2, (3000, F)).astype(np.float32)
    y = (np.sin(X[:, 0]) * X[:, 1] + X[:, 2]).astype(np.float32)
    ds = gg.Dataset(torch.from_numpy(X), torch.from_numpy(y))
    cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    O_op, O_cv = cuda(pop_op), cuda(pop_cv)
    B_op, B_cv = cuda(pop_op), cuda(pop_cv)
    P_op, P_cv = cuda(pop_op), cuda(pop_cv)
    f_b = ds.eval_batch(O_op, O_cv)[0].clone()
    # numpy mirror
    o, c, b, bc = pop_op.copy(), pop_cv.copy(), pop_op.copy(), pop_cv.copy()
    fb = f_b.cpu().numpy().copy()
    heights = np.full(P, h)
    f_new = torch.full((P,), float("nan"), device="cuda")
    for i in range(6):
        donor = rng.integers(0, P, P).astype(np.int32)
        subset = order[:, i].astype(np.int32)
        gg.gom_donate(O_op, O_cv, P_op, P_cv, cuda(donor), cuda(subset), cuda(off), cuda(nodes))
        o, c = gom.donate(o, c, pop_op, pop_cv, donor, subset, fos)
        ch = gg.gom_changed(O_op, O_cv, B_op, B_cv, F)
        ch_ref = gom.changed(o, c, b, bc, heights, "heap", F)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(O_op.cpu().numpy(), o)
        np.testing.assert_array_equal(O_cv.cpu().numpy(), c)
        np.testing.assert_array_equal(ch.cpu().numpy(), ch_ref)
        # evaluate only the changed offspring; the others keep their values
        f_new.fill_(float("nan"))
        ds.eval_batch_masked(O_op, O_cv, ch, out=[f_new, None, None, None])
        fn = f_new.cpu().numpy()
        assert np.all(np.isnan(fn[ch_ref == 0]))
        acc = gg.gom_accept(O_op, O_cv, B_op, B_cv, f_new, f_b, ch)
        o, c, b, bc, fb, acc_ref = gom.accept(o, c, b, bc, ch_ref, fn, fb)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(acc.cpu().numpy(), acc_ref)
        np.testing.assert_array_equal(B_op.cpu().numpy(), b)
        np.testing.assert_array_equal(B_cv.cpu().numpy(), bc)
        np.testing.assert_array_equal(f_b.cpu().numpy(), fb)
    assert acc_ref.sum() > 0 and acc_ref.sum() < P
    ds.sync()
    ds.close()


def test_masked_evaluation_matches_full(gg):
    w = PA.build("c2", 20_000, 200)
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    op, cv = torch.from_numpy(w["op"]).cuda(), torch.from_numpy(w["cval"]).cuda()
    full = ds.eval_batch(op, cv)[0].cpu().numpy()
    mask = (torch.arange(200, device="cuda") % 3 == 0).to(torch.uint8)
    out = torch.full((200,), -1.0, device="cuda")
    ds.eval_batch_masked(op, cv, mask, out=[out, None, None, None])
    got = out.cpu().numpy()
    m = mask.cpu().numpy().astype(bool)
    np.testing.assert_array_equal(got[~m], -1.0)
    np.testing.assert_array_equal(got[m], full[m])
    ds.sync()
    ds.close()
