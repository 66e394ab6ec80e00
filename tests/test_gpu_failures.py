"""Failure detection on the GPU without a GPU fault: the plan's loop-limit test hook
(snd_debug_loop_limit) shrinks the bounds of the bounded device loops (iterations) and waits
(clock cycles), each loop that reaches its bound sets a device status bit and its kernel
returns, snd_candidates reports
SND_ERR_TIMEOUT, and the context stays usable: after the limit is lifted and the workspace
rebound (which clears the status word) the same plan gives the oracle's results again.

Bits (include/snd.h, snd_plan_stats_t.device_status): 16 threshold search, 32 union-find,
128 tree staging wait, 256 grid barrier wait, 512 matched-filter staging wait."""
import pytest

import synth
from oracle import cxx
from oracle import stream as ostream

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_15361_gb300 as g  # noqa: E402

TAU, UNION, TREE_WAIT, GRID_WAIT, MF_WAIT = 16, 32, 128, 256, 512


def _tuples(arr):
    return [(int(c["dm_index"]), int(c["t"]), float(c["snr"]), int(c["width"]), int(c["npix"])) for c in arr]


def _oracle(mode, B):
    w = synth.NC64
    r = cxx.Stream(w.freqs(), synth.NC_DT, w.dms(), ostream.defaults(mode, branching=B)).push(w.chunk_data(0))
    return [(c[0], c[2], float(c[3]), c[4], c[5]) for c in r["candidates"]]


def test_single_plan_loops_time_out_and_recover():
    w = synth.NC64
    chunk = torch.from_numpy(w.chunk_data(0)).cuda()
    plan = g.Plan(w.freqs(), synth.NC_DT, w.dms(), 2, g.MODE_GRADED)
    assert plan.stats().tree_kernel == 1  # the direct kernel with its mbarrier staging waits
    assert g.lib.snd_debug_loop_limit(plan.handle, 1, 1) == 0
    plan.execute(chunk)
    _, rc = plan.candidates(check=False)
    st = plan.stats().device_status
    # the tree's first staging wait gives up (its CTAs stop, so no plane and no islands follow),
    # and so does the matched filter's row staging wait (a bulk copy cannot land in one cycle)
    assert rc == g.ERR["SND_ERR_TIMEOUT"] and st & TREE_WAIT and st & MF_WAIT, (rc, st)
    # lift the limit, rebind (clears the status word): the oracle's candidates again
    assert g.lib.snd_debug_loop_limit(plan.handle, 0, 0) == 0
    plan.bind()
    plan.execute(chunk)
    got, rc = plan.candidates()
    assert rc == 0 and plan.stats().device_status == 0
    assert _tuples(got) == _oracle(g.MODE_GRADED, 2)


def test_batch_grid_barrier_times_out_and_recovers():
    """Two plans in a batch: the cooperative candidate stage's grid barrier takes the first
    plan's bound; a barrier that runs out marks every beam's status word."""
    w = synth.NC64
    chunk = torch.from_numpy(w.chunk_data(0)).cuda()
    plans = [g.Plan(w.freqs(), synth.NC_DT, w.dms(), 2, m) for m in (g.MODE_FLOAT, g.MODE_GRADED)]
    batch = g.Batch(plans)
    assert g.lib.snd_debug_loop_limit(plans[0].handle, 0, 1) == 0
    batch.execute([chunk, chunk])
    _, rc = plans[1].candidates(check=False)
    assert rc == g.ERR["SND_ERR_TIMEOUT"] and plans[1].stats().device_status & GRID_WAIT
    _, rc = plans[0].candidates(check=False)
    assert rc == g.ERR["SND_ERR_TIMEOUT"] and plans[0].stats().device_status & GRID_WAIT
    assert g.lib.snd_debug_loop_limit(plans[0].handle, 0, 0) == 0
    for p in plans:
        p.bind()
    batch = g.Batch(plans)
    batch.execute([chunk, chunk])
    for p, m in zip(plans, (g.MODE_FLOAT, g.MODE_GRADED)):
        got, rc = p.candidates()
        assert rc == 0 and _tuples(got) == _oracle(m, 2)


def test_leaf_sharing_plan_bounds():
    """The leaf-sharing tree has no waits; the union-find walks of a plan with candidates (its
    islands span several DM rows, so several runs) reach a bound of one step (the waits keep
    their default bound, so the matched filter's mask is complete)."""
    w = synth.NC64
    plan = g.Plan(w.freqs(), synth.NC_DT, w.dms(), 2, g.MODE_FLOAT, g.options(g.MODE_FLOAT, flags=g.FLAG_LEAF_SHARING))
    assert g.lib.snd_debug_loop_limit(plan.handle, 1, 0) == 0
    plan.execute(torch.from_numpy(w.chunk_data(0)).cuda())
    _, rc = plan.candidates(check=False)
    st = plan.stats().device_status
    assert not st & TREE_WAIT
    assert st & UNION and rc == g.ERR["SND_ERR_TIMEOUT"], st
