"""Training and evaluation data for the learned sifter, made by the pipeline itself.

A "beam run" is a synthetic Northern Cross beam (1024 channels, 400-416 MHz, dt 0.138 ms,
2048 DMs over 0-2000 pc cm^-3, 16384-sample chunks) with three kinds of injected events:
  * dispersed Gaussian bursts (the positives): DM U(20, 1980), FWHM log-uniform 1-72
    samples, injected S/N log-uniform 5-30;
  * zero-DM broadband impulses: every channel brightened for 1-8 samples;
  * narrowband spikes: 1-16 adjacent channels brightened for 10-500 samples.
The float-mode pipeline (snd_execute, B = 8, detection threshold S/N 5) searches it;
every candidate becomes a standardised 64 x 256 snippet of the float plane (snd_snippets),
labelled positive when it lies within the time and DM tolerance of an injected burst.
The plain sifter's decision is S/N >= 7 (Supplementary Table S1's Theta).

The synthesis runs as torch operations on the GPU (noise, dispersion sweeps and RFI are
input generation); the search and the snippets are the library's kernels.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import MODE_FLOAT, Plan, options, snippets

K_SKY = 4.148808e3
NCHAN, NDM, DM_MAX, CHUNK, DT = 1024, 2048, 2000.0, 16384, 1.38e-4
F_TOP, BW = 416.0, 16.0
PLAIN_THETA = 7.0


@dataclass
class RunData:
    x: "object"        # device float32 [n][64][256] snippets
    label: np.ndarray  # 1 = within tolerance of an injected burst
    snr: np.ndarray    # candidate S/N (the plain sifter's statistic)
    dm_index: np.ndarray
    t: np.ndarray
    kind: np.ndarray   # 0 noise, 1 burst, 2 zero-DM impulse, 3 narrowband spike (nearest event)


def freqs() -> np.ndarray:
    c = np.arange(NCHAN, dtype=np.float64)
    return F_TOP - (c + 0.5) * (BW / NCHAN)


def dm_grid() -> np.ndarray:
    return np.linspace(0.0, DM_MAX, NDM)


def _events(rng, t_hi, n_burst, n_zdm, n_nb):
    """Event times (arrival at the top of the band) in [300, t_hi): the span the search emits
    and scores."""
    bursts = [dict(t0=rng.uniform(300.0, t_hi), dm=rng.uniform(20.0, 1980.0),
                   fwhm=float(np.exp(rng.uniform(0.0, np.log(72.0)))),
                   snr=float(np.exp(rng.uniform(np.log(5.0), np.log(30.0))))) for _ in range(n_burst)]
    zdm = [dict(t=int(rng.integers(300, t_hi)), w=int(rng.integers(1, 9)), amp=rng.uniform(0.5, 3.0))
           for _ in range(n_zdm)]
    nb = [dict(t=int(rng.integers(300, t_hi)), w=int(rng.integers(10, 501)), c0=int(rng.integers(0, NCHAN - 16)),
               nc=int(rng.integers(1, 17)), amp=rng.uniform(2.0, 6.0)) for _ in range(n_nb)]
    return bursts, zdm, nb


def synth_run(seed: int, nchunks: int, n_burst: int, n_zdm: int, n_nb: int, device="cuda"):
    """uint8 device filterbank [nchunks * CHUNK][NCHAN] and its injected events."""
    import torch
    rng = np.random.default_rng([seed, 0x51F7])
    nsamp = nchunks * CHUNK
    f = freqs()
    sweep = K_SKY * DM_MAX * (f.min() ** -2 - f.max() ** -2) / DT
    # plane samples [0, nsamp - D) are emitted, and scored up to Wmax - 1 (<= 1023) before that
    bursts, zdm, nb = _events(rng, nsamp - sweep - 1500.0, n_burst, n_zdm, n_nb)
    gen = torch.Generator(device=device).manual_seed(int(seed))
    x = torch.randn((nsamp, NCHAN), generator=gen, device=device, dtype=torch.float32).mul_(16.0).add_(128.0)
    fd = torch.from_numpy(f).to(device)
    chan = torch.arange(NCHAN, device=device)
    for b in bursts:
        sig_t = b["fwhm"] / 2.3548
        half = int(math.ceil(4.0 * sig_t)) + 1
        arr = b["t0"] + K_SKY * b["dm"] * (fd ** -2 - F_TOP ** -2) / DT          # [nchan], samples
        base = torch.floor(arr).long()
        off = torch.arange(-half, half + 1, device=device)
        tt = base[:, None] + off[None, :]                                      # [nchan][win]
        gprof = torch.exp(-0.5 * ((tt.double() - arr[:, None]) / sig_t) ** 2)
        amp = b["snr"] / math.sqrt(NCHAN * float((gprof ** 2).sum() / NCHAN))
        ok = (tt >= 0) & (tt < nsamp)
        x.index_put_((tt[ok], chan[:, None].expand_as(tt)[ok]), (16.0 * amp * gprof[ok]).float(), accumulate=True)
    for z in zdm:
        x[z["t"]:z["t"] + z["w"], :] += 16.0 * z["amp"]
    for q in nb:
        x[q["t"]:q["t"] + q["w"], q["c0"]:q["c0"] + q["nc"]] += 16.0 * q["amp"]
    data = x.round_().clamp_(0, 255).to(torch.uint8)
    return data, dict(bursts=bursts, zdm=zdm, nb=nb)


def search_run(data, nchunks: int, theta: float = 5.0, device="cuda"):
    """Float-mode search of a synthetic run: candidates (structured array) and the float
    plane [NDM][E] of every emitted sample."""
    import torch
    opts = options(MODE_FLOAT, det_theta=theta, max_chunk=CHUNK)
    plan = Plan(freqs(), DT, dm_grid(), 8, MODE_FLOAT, opts, device=device)
    D = plan.stats().max_delay
    total_e = nchunks * CHUNK - D
    plane = torch.zeros((NDM, max(total_e, 1)), dtype=torch.float32, device=device)
    out = torch.empty(NDM * CHUNK, dtype=torch.float32, device=device)  # [NDM][nemit] per call
    e = 0
    for i in range(nchunks):
        ne = plan.execute(data[i * CHUNK:(i + 1) * CHUNK], out)
        if ne:
            plane[:, e:e + ne] = out[:NDM * ne].view(NDM, ne)
            e += ne
    cands, _ = plan.candidates(check=False)
    return cands, plane[:, :e]


def label_candidates(cands, events):
    """1 for candidates near an injected burst (|dt| <= max(64, 3 FWHM) samples and
    |dDM| <= max(30, 0.15 DM)), plus the kind of the nearest event in time."""
    dms = dm_grid()
    lab = np.zeros(len(cands), dtype=np.int64)
    kind = np.zeros(len(cands), dtype=np.int64)
    for i, c in enumerate(cands):
        t, dm = int(c["t"]), dms[int(c["dm_index"])]
        for b in events["bursts"]:
            if abs(t - b["t0"]) <= max(64.0, 3.0 * b["fwhm"]) and abs(dm - b["dm"]) <= max(30.0, 0.15 * b["dm"]):
                lab[i] = 1
                kind[i] = 1
                break
        if lab[i]:
            continue
        best = 1e18
        for z in events["zdm"]:
            if abs(t - z["t"]) < best and abs(t - z["t"]) <= 600:
                best, kind[i] = abs(t - z["t"]), 2
        for q in events["nb"]:
            d = min(abs(t - q["t"]), abs(t - q["t"] - q["w"]))
            if d < best and (q["t"] - 600 <= t <= q["t"] + q["w"] + 600):
                best, kind[i] = d, 3
    return lab, kind


def make_run(seed: int, nchunks: int = 6, n_burst: int = 48, n_zdm: int = 16, n_nb: int = 16,
             device="cuda") -> RunData:
    import torch
    data, ev = synth_run(seed, nchunks, n_burst, n_zdm, n_nb, device)
    cands, plane = search_run(data, nchunks, device=device)
    del data
    lab, kind = label_candidates(cands, ev)
    rows = torch.from_numpy(cands["dm_index"].astype(np.int32)).to(device)
    cols = torch.from_numpy(cands["t"].astype(np.int64)).to(device)
    x = snippets(plane, rows, cols) if len(cands) else torch.zeros((0, 64, 256), device=device)
    return RunData(x, lab, cands["snr"].astype(np.float64), cands["dm_index"].astype(np.int64),
                   cands["t"].astype(np.int64), kind)


def concat(runs) -> RunData:
    import torch
    return RunData(torch.cat([r.x for r in runs]), np.concatenate([r.label for r in runs]),
                   np.concatenate([r.snr for r in runs]), np.concatenate([r.dm_index for r in runs]),
                   np.concatenate([r.t for r in runs]), np.concatenate([r.kind for r in runs]))


def train(sifter, data: RunData, epochs: int = 3, batch: int = 256, lr: float = 1e-3, seed: int = 0):
    """Adam on the GPU over shuffled batches; returns the mean loss of each epoch."""
    import torch
    n = data.x.shape[0]
    y = torch.from_numpy(data.label.astype(np.float32)).to(data.x.device)
    loss = torch.zeros(1, device=data.x.device)
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).to(data.x.device)
        tot = 0.0
        nb = 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            sifter.train_step(data.x[idx].contiguous(), y[idx].contiguous(), lr, loss)
            tot += float(loss.item()) if nb % 50 == 0 else 0.0
            nb += 1
        sifter.status()
        out.append(tot / max(1, (nb + 49) // 50))
    return out


def logits(sifter, x, batch: int):
    import torch
    out = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    for s in range(0, x.shape[0], batch):
        sifter.forward(x[s:s + batch].contiguous(), out[s:s + batch])
    return out.cpu().numpy().astype(np.float64)


def compare(scores: np.ndarray, data: RunData) -> dict:
    """Miss rate of the learned sifter at the plain sifter's false-alarm rate on `data`."""
    pos, neg = data.label == 1, data.label == 0
    plain = data.snr >= PLAIN_THETA
    far_plain = float(plain[neg].mean()) if neg.any() else 0.0
    miss_plain = float((~plain[pos]).mean()) if pos.any() else 0.0
    # the learned threshold that accepts the same fraction of negatives
    sneg = np.sort(scores[neg])[::-1]
    k = int(math.floor(far_plain * len(sneg)))
    thr = sneg[k] if k < len(sneg) else -np.inf  # accept scores strictly above the (k+1)-th best negative
    acc = scores > thr
    far_cnn = float(acc[neg].mean()) if neg.any() else 0.0
    miss_cnn = float((~acc[pos]).mean()) if pos.any() else 0.0
    by_kind = {name: dict(n=int((data.kind == k).sum()), plain_accept=float(plain[data.kind == k].mean())
                          if (data.kind == k).any() else None,
                          learned_accept=float(acc[data.kind == k].mean()) if (data.kind == k).any() else None)
               for k, name in ((0, "noise"), (1, "burst"), (2, "zero_dm"), (3, "narrowband"))}
    return dict(n=int(len(scores)), positives=int(pos.sum()), negatives=int(neg.sum()), far_plain=far_plain,
                miss_plain=miss_plain, far_learned=far_cnn, miss_learned=miss_cnn, threshold=float(thr),
                by_kind=by_kind)
