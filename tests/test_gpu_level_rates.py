"""Per-level fire counts (SND_FLAG_LEVEL_RATES, snd_level_rates) against the oracle's
oracle.tree.level_fire_counts on the same encoded stream: for every tree level, the number of
node-samples with a nonzero output over all emitted samples and DM rows must be equal. Binary
plans count in the tree kernel itself (also in a batch, through the persistent kernel); float
and graded plans through the binary counting pass with K_L = K_I = 1 (a node is nonzero iff a
channel of its subtree fired)."""
import numpy as np
import pytest

import synth
from oracle import delays as odelays
from oracle import encoder as oenc
from oracle import stream as ostream
from oracle import tree as otree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_15361_gb300 as g  # noqa: E402


def _oracle_counts(freqs, dms, chunks, cfg):
    tab = odelays.delay_table(freqs, synth.NC_DT, dms)
    D = int(tab.max())
    x = np.concatenate([oenc.encode_chunk(c, cfg.enc_theta)[0] for c in chunks], axis=1)
    n = x.shape[1] - D
    return otree.level_fire_counts(x, 0, tab, range(len(dms)), 0, n, cfg.mode, cfg.cluster, cfg.branching,
                                   cfg.k_leaf, cfg.k_internal, cfg.cap), n


CASES = [("binary", 8, 64, 128, 100.0), ("binary", 2, 64, 128, 100.0), ("float", 8, 64, 128, 100.0),
         ("graded", 2, 64, 128, 100.0), ("float", 8, 1024, 40, 600.0), ("binary", 4, 1024, 40, 600.0)]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-B{c[1]}-{c[2]}ch" for c in CASES])
def test_level_fire_counts_match_oracle(case):
    mode_name, B, nchan, ndm, dm_max = case
    m = {"binary": ostream.BINARY, "graded": ostream.GRADED, "float": ostream.FLOAT}[mode_name]
    freqs, dms = synth.channel_freqs(nchan), synth.dm_grid(ndm, dm_max)
    D = int(odelays.delay_table(freqs, synth.NC_DT, dms).max())
    n = D + 5000
    data = synth.filterbank_chunk(33, 0, 0, n, freqs, synth.NC_DT, [synth.Burst(2000.0, 0.5 * dm_max, 8.0, 40.0)])
    chunks = [data[: n // 2], data[n // 2:]]
    cfg = ostream.defaults(m, branching=B)
    plan = g.Plan(freqs, synth.NC_DT, dms, B, m, g.options(m, flags=g.FLAG_LEVEL_RATES))
    assert plan.stats().tree_kernel == 1
    for c in chunks:
        plan.execute(torch.from_numpy(np.ascontiguousarray(c)).cuda())
    fires, rates = plan.level_rates()
    want, nout = _oracle_counts(freqs, dms, chunks, cfg)
    assert [int(f) for f in fires] == want
    lv = otree.tree_levels(nchan, 4, B)
    for l in range(len(lv)):
        assert rates[l] == pytest.approx(want[l] / (len(lv[l]) * ndm * nout))


def test_binary_counts_in_a_batch():
    freqs, dms = synth.channel_freqs(64), synth.dm_grid(128, 100.0)
    data = synth.NC64.chunk_data(0)
    plans = [g.Plan(freqs, synth.NC_DT, dms, 2, g.MODE_BINARY, g.options(g.MODE_BINARY, flags=g.FLAG_LEVEL_RATES))
             for _ in range(2)]
    batch = g.Batch(plans)
    for a, b in ((0, 7000), (7000, 16384)):
        c = torch.from_numpy(np.ascontiguousarray(data[a:b])).cuda()
        batch.execute([c, c])
    want, _ = _oracle_counts(freqs, dms, [data[:7000], data[7000:]], ostream.defaults(ostream.BINARY, branching=2))
    for p in plans:
        assert [int(f) for f in p.level_rates()[0]] == want


def test_flag_rejected_where_the_counting_kernel_does_not_apply():
    freqs, dms = synth.channel_freqs(96), synth.dm_grid(16, 50.0)   # 96 channels: not a multiple of 64
    with pytest.raises(g.SndError) as e:
        g.Plan(freqs, synth.NC_DT, dms, 2, g.MODE_FLOAT, g.options(g.MODE_FLOAT, flags=g.FLAG_LEVEL_RATES), bind=False)
    assert e.value.code == g.ERR["SND_ERR_UNSUPPORTED"]
