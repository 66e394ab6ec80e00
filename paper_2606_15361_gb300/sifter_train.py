"""Train the learned sifter on snippets made by the pipeline and compare it with the plain
sifter at equal false-alarm rate.

    python -m paper_2606_15361_gb300.sifter_train --train-snippets 200000 --epochs 6

Prints one JSON object: data sizes and generation time, the loss per epoch, training and
inference throughput, and the comparison (false-alarm and miss rates, acceptance by event
kind). --save writes the trained parameter vector (float32 .npy).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main(argv=None):
    import torch

    from . import Sifter
    from . import sifter_data as sd

    ap = argparse.ArgumentParser()
    ap.add_argument("--train-snippets", type=int, default=200000)
    ap.add_argument("--test-runs", type=int, default=60)
    ap.add_argument("--bursts-per-run", type=int, default=96)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--infer-batch", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--save", default=None)
    a = ap.parse_args(argv)

    t0 = time.perf_counter()
    runs, n, s = [], 0, 0
    while n < a.train_snippets:
        r = sd.make_run(100000 * a.seed + s, n_burst=a.bursts_per_run)
        runs.append(r)
        n += len(r.label)
        s += 1
    tr = sd.concat(runs)
    del runs
    te = sd.concat([sd.make_run(900000 + 1000 * a.seed + i, n_burst=a.bursts_per_run) for i in range(a.test_runs)])
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0

    sf = Sifter(max_batch=a.batch, training=True, seed=a.seed)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    losses = sd.train(sf, tr, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed)
    ev1.record()
    torch.cuda.synchronize()
    train_s = ev0.elapsed_time(ev1) / 1e3
    steps = a.epochs * (len(tr.label) // a.batch)

    inf = Sifter(max_batch=a.infer_batch, training=False, seed=a.seed)
    inf.set_params(sf.get_params())
    scores = sd.logits(inf, te.x, a.infer_batch)
    xb = te.x[:a.infer_batch].contiguous() if te.x.shape[0] >= a.infer_batch else \
        te.x.repeat((a.infer_batch + te.x.shape[0] - 1) // te.x.shape[0], 1, 1)[:a.infer_batch].contiguous()
    for _ in range(3):
        inf.forward(xb)
    ev0.record()
    for _ in range(10):
        inf.forward(xb)
    ev1.record()
    torch.cuda.synchronize()
    infer_ms = ev0.elapsed_time(ev1) / 10
    out = dict(train_snippets=int(len(tr.label)), train_positives=int(tr.label.sum()), train_runs=s,
               test_snippets=int(len(te.label)), test_positives=int(te.label.sum()), data_seconds=round(t_data, 1),
               epochs=a.epochs, batch=a.batch, lr=a.lr, loss_per_epoch=[round(x, 4) for x in losses],
               train_snippets_per_s=round(steps * a.batch / train_s, 1),
               infer_batch=a.infer_batch, infer_ms_per_batch=round(infer_ms, 3),
               infer_snippets_per_s=round(a.infer_batch / (infer_ms / 1e3), 1),
               comparison=sd.compare(scores, te))
    if a.save:
        np.save(a.save, sf.get_params())
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
