"""snd_encode_static: the encoder entry point that needs no device allocation (for callers
that cannot call cudaMalloc). Its spike raster must equal the one the regular streaming
entry point (snd_execute) produces. With one channel, one trial DM of 0 and float mode the
plane snd_execute writes is exactly the channel's spike train (the tree is a single leaf,
the delay is 0 and 1/sqrt(N_f) = 1), so every channel is checked against its own
single-channel plan, and against the oracle's encoder (oracle.encoder.encode_chunk). Two calls
in a row, on different chunks, check that the shared scratch starts clean each time. The
largest accepted channel count (4096, whose histogram fills the scratch up to the levels) and
a multiple of 32 over several channel blocks are covered too. This file is collected last on
purpose."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import encoder as oenc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_15361_gb300 as g  # noqa: E402


def _encode_static(chunk: torch.Tensor, theta: float) -> np.ndarray:
    nsamp, nchan = chunk.shape
    nwords = (nsamp + 31) // 32
    bits = torch.zeros((nchan, nwords), dtype=torch.int32, device="cuda")
    rc = g.lib.snd_encode_static(ctypes.c_void_p(chunk.data_ptr()), nsamp, nchan, theta,
                                 ctypes.c_void_p(bits.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, g.STATUS.get(rc, rc)
    torch.cuda.synchronize()
    w = bits.cpu().numpy().view(np.uint32)
    return ((w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(nchan, -1)[:, :nsamp].astype(bool)


def _execute_single_channel(col: np.ndarray, theta: float) -> np.ndarray:
    nsamp = col.size
    opts = g.options(g.MODE_FLOAT, cluster_size=1, enc_theta=theta, max_chunk=nsamp)
    plan = g.Plan(np.array([400.0]), synth.NC_DT, np.array([0.0]), 2, g.MODE_FLOAT, opts)
    out = torch.empty((1, nsamp), dtype=torch.float32, device="cuda")
    assert plan.execute(torch.from_numpy(np.ascontiguousarray(col[:, None])).cuda(), out) == nsamp
    return out.cpu().numpy()[0] == 1.0


@pytest.mark.parametrize("theta", [1.5, 0.75])
def test_encode_static_matches_execute(theta):
    nchan = 40
    freqs = synth.channel_freqs(nchan)
    for call, nsamp in enumerate((3000, 4111)):
        bursts = [synth.Burst(600.0 + 500 * call, 5.0, 8.0, 60.0)]
        data = synth.filterbank_chunk(90 + call, 0, 0, nsamp, freqs, synth.NC_DT, bursts)
        data[:, 3] = 77          # constant channel: never fires
        data[::7, 5] = 255       # heavy tail: the sigma clip matters
        got = _encode_static(torch.from_numpy(data).cuda(), theta)
        assert got.shape == (nchan, nsamp)
        assert not got[3].any()
        for c in range(nchan):
            assert (got[c] == _execute_single_channel(data[:, c], theta)).all(), (call, c)
        assert (got == oenc.encode_chunk(data, theta)[0]).all()


@pytest.mark.parametrize("nchan,nsamp", [(96, 2500), (4096, 300)])
def test_encode_static_channel_blocks_and_largest_size(nchan, nsamp):
    """96 channels: three full 32-channel blocks; 4096: the largest accepted, its histogram
    ends where the levels begin. Two calls in a row; every channel against the oracle, a
    spread of channels (the last ones included) against single-channel snd_execute plans."""
    freqs = synth.channel_freqs(nchan)
    for call in range(2):
        data = synth.filterbank_chunk(70 + call, 0, 0, nsamp, freqs, synth.NC_DT, [])
        data[::5, -1] = 250
        got = _encode_static(torch.from_numpy(data).cuda(), 1.5)
        assert (got == oenc.encode_chunk(data, 1.5)[0]).all()
        for c in sorted({0, 31, 32, nchan // 2, nchan - 2, nchan - 1}):
            assert (got[c] == _execute_single_channel(data[:, c], 1.5)).all(), (call, c)


def test_encode_static_rejects_sizes_beyond_its_limits():
    chunk = torch.zeros((64, 4097), dtype=torch.uint8, device="cuda")
    bits = torch.zeros((4097, 2), dtype=torch.int32, device="cuda")
    rc = g.lib.snd_encode_static(ctypes.c_void_p(chunk.data_ptr()), 64, 4097, 1.5, ctypes.c_void_p(bits.data_ptr()),
                                 None)
    assert rc == g.ERR["SND_ERR_UNSUPPORTED"]
    # too many samples: rejected before any work is enqueued, so the (small) buffers are
    # never read or written
    rc = g.lib.snd_encode_static(ctypes.c_void_p(chunk.data_ptr()), 65535 * 256 + 1, 1, 1.5,
                                 ctypes.c_void_p(bits.data_ptr()), None)
    assert rc == g.ERR["SND_ERR_UNSUPPORTED"]
