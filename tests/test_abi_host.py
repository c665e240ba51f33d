"""CPU tests of the C-ABI library: it loads, exports every symbol the header
declares, its opcode values match the interface, and its packer (run on the
host through ggeval_pack_host / ggeval_batch_stats) linearises templates to
programs that compute the oracle's value.  No GPU is touched."""
import os
import re

import numpy as np
import pytest
import torch

import oracle as O
import synth
from fixtures import fig1, heap_template
import isa_emulator as emu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ggeval.h")


@pytest.fixture(scope="module")
def gg():
    import paper_2605_30954_gb300 as pkg
    if not os.path.exists(pkg.ggeval.LIB_PATH):
        try:
            pkg.build()
        except RuntimeError as e:  # no nvcc on this machine
            pytest.skip(f"cannot build the library: {e}")
    return pkg


def header_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(ggeval_[a-z_]+)\s*\(", text)))


def test_library_exports_every_header_symbol(gg):
    lib = gg.lib()
    names = header_functions()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(gg.ggeval.SYMBOLS)
    assert b"sm_103a" in lib.ggeval_version()


def test_header_opcodes_match_interface():
    text = open(HEADER).read()
    vals = dict((k, int(v)) for k, v in re.findall(r"GGEVAL_OP_([A-Z0-9_]+)\s*=\s*(\d+)", text))
    names = {"ADD": "ADD", "SUB": "SUB", "MUL": "MUL", "AQ": "AQ", "SIN": "SIN", "COS": "COS",
             "EXP": "EXP", "LOG_ABS": "LOG_ABS", "SQRT_ABS": "SQRT_ABS", "DIV": "DIV",
             "SQUARE": "SQUARE", "LOG": "LOG", "SQRT": "SQRT", "POW": "POW", "ERC": "ERC",
             "FEATURE0": "FEAT0",
             "PAD": "PAD"}
    for h, o in names.items():
        assert vals[h] == getattr(O, o) == getattr(synth, o), h


def pack(gg, op, cv, h, layout=0, nf=8):
    opt = torch.from_numpy(np.ascontiguousarray(op[None]))
    cvt = torch.from_numpy(np.ascontiguousarray(cv[None]))
    hs = torch.tensor([h], dtype=torch.int8)
    stride = op.shape[0]
    maxh = (stride + 1).bit_length() - 2
    b = gg.make_batch(opt, cvt, hs if h != maxh else None, layout=layout)
    return gg.pack_host(opt, cvt, 0, hs if h != maxh else None, layout=layout, n_features=nf)


def test_fig1_program(gg):
    op, cv, rows = fig1()
    words, consts, tpos = pack(gg, op, cv, 3, nf=6)
    # the figure's RPN "-2 4 x0 * x1 + /" with each terminal fused into its
    # parent where possible: 4 x0 * | x1 + | -2 (left operand) /
    assert emu.tokens(words, consts) == ["ldc 4", "bf * x0", "bf + x1", "lc / -2"]
    assert list(tpos) == [11, 5, 2, 0]
    X = np.random.default_rng(0).uniform(1, 2, (50, 6))
    val, slots = emu.run(words, consts, X)
    np.testing.assert_allclose(val, -2.0 / (4.0 * X[:, 0] + X[:, 1]), rtol=1e-15)
    assert slots == 0


@pytest.mark.parametrize("layout", ["heap", "prefix"])
@pytest.mark.parametrize("h", [0, 1, 2, 3, 4, 5, 6, 7, 8])
def test_packed_programs_compute_the_oracle_value(gg, h, layout):
    rng = np.random.default_rng(100 + h)
    nf = 5
    X = rng.uniform(-2, 2, (40, nf))
    funcs = synth.FULL_SET + (synth.DIV, synth.SQUARE, synth.POW)
    for p_func in (0.5, 1.0):
        op, cv, hs = synth.random_templates(rng, 12, h, h, funcs, nf, p_func)
        if layout == "prefix":
            op, cv = synth.to_prefix(op, cv, hs.astype(np.int64))
        for p in range(op.shape[0]):
            words, consts, tpos = pack(gg, op[p], cv[p], h, 0 if layout == "heap" else 1, nf)
            t = O.Template(op[p], cv[p], h, layout, nf)
            want = O.eval_tree(t, X)
            got, slots = emu.run(words, consts, X)
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-300, equal_nan=True)
            assert slots <= max(h - 1, 0)
            assert len(words) <= int(O.active_mask(t).sum())
            # a load without a push comes first and nowhere else (the
            # interpreter decides the first instruction before its switch)
            opc = np.asarray(words) & 0xFF
            assert opc[0] in (emu.I_LDF0, emu.I_LDC0)
            assert not np.isin(opc[1:], (emu.I_LDF0, emu.I_LDC0)).any()


def folded_nodes(t):
    """(nodes strictly below the roots of maximal feature-free active
    subtrees, number of such roots that are functions)."""
    out = [0, 0]

    def const(pos, d):  # -> (no feature below, active size)
        o = int(t.op[pos])
        if o >= synth.FEAT0 and o != synth.PAD:
            return False, 1
        if o == synth.ERC:
            return True, 1
        l, r = t.children(pos, d)
        parts = [const(l, d + 1)] + ([const(r, d + 1)] if o in synth.BINARY else [])
        c = all(x[0] for x in parts)
        if not c:
            for pc, pn in parts:
                if pc and pn > 1:
                    out[0] += pn - 1
                    out[1] += 1
        return c, 1 + sum(x[1] for x in parts)

    c, n = const(0, 0)
    if c and n > 1:
        out[0] += n - 1
        out[1] += 1
    return out[0], out[1]


def test_stats_count_active_nodes(gg):
    rng = np.random.default_rng(3)
    op, cv, hs = synth.random_templates(rng, 50, rng.integers(0, 6, 50), 5,
                                        synth.FULL_SET + (synth.POW,), 4, 0.7)
    st = gg.batch_stats(torch.from_numpy(op), torch.from_numpy(cv),
                        torch.from_numpy(hs), n_features=4).numpy()
    total_removed = 0
    for p in range(50):
        t = O.Template(op[p], cv[p], int(hs[p]), n_features=4)
        mask = O.active_mask(t)
        assert st[p, 0] == mask.sum()
        assert st[p, 1] == np.sum(mask & (op[p] >= synth.ERC))
        assert st[p, 0] == st[p, 1:10].sum() + st[p, 12]
        assert st[p, 12] == np.sum(mask & (op[p] == synth.POW))
        # constant folding: every active subtree without a feature becomes one
        # constant terminal (structure counted here by a plain recursion)
        removed, roots = folded_nodes(t)
        total_removed += removed
        assert st[p, 13] == st[p, 0] - removed and st[p, 14] >= roots
        assert st[p, 13] == st[p, 14:23].sum() + st[p, 23]
        assert st[p, 24] <= st[p, 10]
    assert total_removed > 10  # the batch has constant subtrees to fold


@pytest.mark.parametrize("tokens,h", [
    (["+", "x0", "*"], 1),        # function at a leaf position, active
    (["+", "x0", None], 1),       # PAD active
    (["+", "x0", "x9"], 1),       # feature index >= n_features
    ([None], 0),
])
def test_invalid_templates_rejected(gg, tokens, h):
    op, cv = heap_template(tokens, h)
    with pytest.raises(gg.GGEvalError) as e:
        pack(gg, op, cv, h, nf=4)
    assert e.value.status == -2


def test_intron_function_at_leaf_is_accepted(gg):
    op, cv = heap_template(["+", "x0", "x1", "*", "sin", "exp", None], 2)
    words, consts, _ = pack(gg, op, cv, 2, nf=2)
    assert emu.tokens(words, consts) == ["ldf x0", "bf + x1"]
