"""The device packer (one warp per trial, level-parallel) against the host
packer (sequential): identical programs for every height, both layouts and
every operator when folding is off; with folding on, the program lengths
the host's structural count predicts, and programs whose FP64 emulation
tracks the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
import isa_emulator as emu

pytestmark = pytest.mark.gpu

FUNCS = synth.FULL_SET + (synth.DIV, synth.SQUARE, synth.LOG, synth.SQRT, synth.POW)
NF = 5


@pytest.fixture(scope="module")
def gg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_30954_gb300 as pkg
    pkg.lib()
    return pkg


def batch(rng, n, h_max, p_func, layout):
    hs = rng.integers(0, h_max + 1, n) if h_max else np.zeros(n, dtype=np.int64)
    op, cv, hs = synth.random_templates(rng, n, hs, h_max, FUNCS, NF, p_func)
    if layout == "prefix":
        op, cv = synth.to_prefix(op, cv, hs.astype(np.int64))
    return op, cv, hs.astype(np.int8)


@pytest.mark.parametrize("layout", ["heap", "prefix"])
def test_device_programs_equal_host_programs(gg, layout):
    rng = np.random.default_rng(11)
    X = rng.uniform(0.5, 2.0, (64, NF)).astype(np.float32)
    ds = gg.Dataset(torch.from_numpy(X), torch.from_numpy(X[:, 0].copy()))
    lay = 0 if layout == "heap" else 1
    checked = 0
    for h_max in (0, 1, 2, 3, 4, 5, 6, 7, 8):
        for p_func in (0.5, 0.95):
            op, cv, hs = batch(rng, 48, h_max, p_func, layout)
            args = (torch.from_numpy(op).cuda(), torch.from_numpy(cv).cuda(),
                    torch.from_numpy(hs).cuda())
            w, c, L = ds.pack_device(*args, layout=lay, flags=gg.F_POW | gg.F_NO_FOLD)
            for p in range(op.shape[0]):
                hw, hc, _ = gg.pack_host(torch.from_numpy(op), torch.from_numpy(cv), p,
                                         torch.from_numpy(hs), layout=lay, n_features=NF)
                assert L[p] == len(hw), (h_max, p)
                np.testing.assert_array_equal(w[p, :L[p]], hw)
                np.testing.assert_array_equal(c[p, :L[p]].view(np.uint32), hc.view(np.uint32))
                checked += 1
    ds.sync()
    ds.close()
    assert checked == 2 * 9 * 48


@pytest.mark.parametrize("layout", ["heap", "prefix"])
def test_folded_programs(gg, layout):
    rng = np.random.default_rng(12)
    X = rng.uniform(0.5, 2.0, (64, NF)).astype(np.float32)
    X64 = X.astype(np.float64)
    ds = gg.Dataset(torch.from_numpy(X), torch.from_numpy(X[:, 0].copy()))
    lay = 0 if layout == "heap" else 1
    shorter = compared = 0
    for h_max in (2, 3, 4, 6):
        op, cv, hs = batch(rng, 64, h_max, 0.6, layout)
        args = (torch.from_numpy(op).cuda(), torch.from_numpy(cv).cuda(),
                torch.from_numpy(hs).cuda())
        w, c, L = ds.pack_device(*args, layout=lay, flags=gg.F_POW)
        st = gg.batch_stats(torch.from_numpy(op), torch.from_numpy(cv), torch.from_numpy(hs),
                            layout=lay, n_features=NF).numpy()
        np.testing.assert_array_equal(L, st[:, 24])
        shorter += int(np.sum(st[:, 24] < st[:, 10]))
        for p in range(op.shape[0]):  # a load without a push first, and only there
            if L[p] <= 0:
                continue
            opc = w[p, :L[p]] & 0xFF
            assert opc[0] in (emu.I_LDF0, emu.I_LDC0)
            assert not np.isin(opc[1:], (emu.I_LDF0, emu.I_LDC0)).any()
        if h_max > 4:
            continue
        for p in range(op.shape[0]):
            t = O.Template(op[p], cv[p], int(hs[p]), layout, NF)
            want = O.eval_tree(t, X64)
            got, _ = emu.run(w[p, :L[p]], c[p, :L[p]], X64)
            with np.errstate(all="ignore"):
                ok = np.isfinite(want) & (np.abs(want) < 1e4)
            if ok.all():  # folded constants are FP32 values: compare loosely
                np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-4)
                compared += 1
    ds.sync()
    ds.close()
    assert shorter > 20 and compared > 100
