"""GPU parity of deferred validation -- several kernel rounds checked in one
launch, as no-sync sessions with PHOS_CKPT_DEFER run it -- against the
oracle, through phos_harness_validate_rounds.

Per round the oracle's validation (Sec. 4.1, linear scan) gives the store
victims and the victims of any access; each protocol's response then fixes
the result: recopy (Sec. 4.3) marks every store victim the copier had
touched dirty, CoW (Sec. 4.2) calls a round with a store victim that is
neither done nor shadowed a mis-speculation, restore (Sec. 6) a round with
any victim not restored.  Compared exactly: the dirty set, the first
mis-speculated round (device word and the flag word) and the violation
count, on two launches in a row over the same scratch.

Shapes: long rounds (the training step's ~10^6 records per kernel; the
launch takes 32-word batches and prefetches), short rounds (8-word
batches), and a mix of long rounds with rounds of 1 to 777 records (partial
batches next to full ones), each with ragged lengths.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core  # noqa: E402
from paper_2405_12079_b300 import phos, workloads as wl  # noqa: E402
from gpu_util import dev, host, stream  # noqa: E402

VA0 = 0x7E00_0000_0000
RULE_RECOPY, RULE_COW, RULE_RESTORE = 1, 2, 3


def round_lengths(shape, rng):
    if shape == "long":
        return [int(x) for x in rng.integers(500_000, 700_000, 16)]
    if shape == "short":
        return [int(x) for x in rng.integers(1, 20_000, 16)]
    return [1, 2_000_003, 40, 1_500_001, 65_536, 777]


def make_rounds(shape, n_buf, seed, covered_rounds):
    """Random table, then per round: read/write sets, the perms speculation
    gives them, a coalesced trace with strays (30 % stores), and rule flags
    (every buffer covered for the first `covered_rounds` rounds, random
    after)."""
    rng = np.random.default_rng(seed)
    lay = wl.make_layout(rng, wl.sizes_uniform(rng, n_buf, 256, 1 << 20))
    base = lay.base(VA0)
    rounds = []
    for i, n_rec in enumerate(round_lengths(shape, rng)):
        reads, writes = wl.pick_sets(rng, n_buf, 1, 20)
        perm = np.zeros(n_buf, np.uint8)
        perm[reads] = phos.PERM_R
        perm[writes] = phos.PERM_RW
        rec, _, _ = wl.trace_runs(rng, lay, VA0, reads, writes, n_rec, stray_frac=0.002,
                                  stray_store_frac=0.3)
        flags = (np.ones(n_buf, np.uint8) if i < covered_rounds
                 else (rng.random(n_buf) < 0.5).astype(np.uint8))
        rounds.append(dict(rec=rec, perm=perm, flags=flags, round=1000 + 7 * i))
    return lay, base, rounds


def bits(words, n):
    return np.unpackbits(np.asarray(words, np.uint32).view(np.uint8),
                         bitorder="little")[:n].astype(bool)


_CASES = {}


def world(shape, covered):
    """Table, rounds and the oracle's validation of each round (computed
    once per shape and shared by the three rules)."""
    key = (shape, covered)
    if key not in _CASES:
        lay, base, rounds = make_rounds(shape, 1000, 4242 + len(shape) + covered, covered)
        for r in rounds:
            r["oracle"] = core.validate(base, lay.size, r["perm"], r["rec"], 4)
        _CASES.clear()
        _CASES[key] = (lay, base, rounds)
    return _CASES[key]


def expected(base, rounds, rule):
    """The protocol's response to the oracle's validation of each round."""
    n = len(base)
    dirty = np.zeros(n, bool)
    viol, first = 0, -1
    for r in rounds:
        e = r["oracle"]
        viol += int(e.count[0])
        vic = bits(e.victim if rule == RULE_RESTORE else e.victim_st, n)
        covered = r["flags"] != 0
        if rule == RULE_RECOPY:
            dirty |= vic & covered
        elif first < 0 and (vic & ~covered).any():
            first = r["round"]
    return dirty, viol, first


@pytest.mark.parametrize("rule", [RULE_RECOPY, RULE_COW, RULE_RESTORE])
@pytest.mark.parametrize("shape,covered", [("long", 5), ("short", 3), ("mixed", 2),
                                           ("long", 16)])
def test_deferred_rounds_equal_oracle(shape, covered, rule):
    n_buf = 1000
    lay, base, rounds = world(shape, covered)
    t = phos.Table(base, lay.size)
    scratch_bytes, max_rounds = phos.harness_rounds_scratch(t)
    assert max_rounds >= len(rounds)
    keep = []
    spec = []
    for r in rounds:
        d_tr, d_pm, d_fl = dev(r["rec"]), dev(r["perm"]), dev(r["flags"])
        keep += [d_tr, d_pm, d_fl]
        spec.append((d_tr.data_ptr(), len(r["rec"]), d_pm.data_ptr(), d_fl.data_ptr(),
                     r["round"]))
    d_dirty = torch.zeros(n_buf, dtype=torch.uint8, device="cuda")
    acc0 = np.array([0, 0, 0, 0, 2**64 - 1, 0, 0, 0], np.uint64)
    d_acc = dev(acc0)
    d_flag = dev(np.array([-1], np.int64))
    d_st = torch.zeros(4, dtype=torch.uint8, device="cuda")
    d_scr = torch.zeros(scratch_bytes, dtype=torch.uint8, device="cuda")
    exp_dirty, exp_viol, exp_first = expected(base, rounds, rule)
    for call in (1, 2):
        phos.harness_validate_rounds(t, spec, 4, rule, d_dirty.data_ptr(), d_acc.data_ptr(),
                                     d_flag.data_ptr(), d_st.data_ptr(), d_scr.data_ptr(),
                                     stream())
        torch.cuda.synchronize()
        acc = host(d_acc, np.uint64)
        assert int(acc[3]) == call * exp_viol
        assert host(d_st, np.uint32)[0] == 0
        assert np.array_equal(host(d_dirty, np.uint8).astype(bool), exp_dirty)
        first = int(acc[4].astype(np.int64))
        assert first == exp_first
        assert int(host(d_flag, np.int64)[0]) == exp_first
        # the launch leaves its scratch zeroed
        assert not host(d_scr, np.uint8).any()
    assert exp_viol > 0
    if rule == RULE_RECOPY:
        assert exp_dirty.any()
    elif covered < len(rounds):
        # a mis-speculation, and not before the first round with gaps in
        # its flags
        assert exp_first >= rounds[covered]["round"]
