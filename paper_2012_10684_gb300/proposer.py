"""Training of the learned threshold proposer, on the GPU, through the C ABI.

Data: seeded chest phantoms (512 x 512 x D, D uniform in [dmin, dmax], sensor
noise sd uniform in [5, 30] HU, 4-8 airway generations), generated on the
GPU one at a time. For each volume the 4096-level whole-volume histogram and
the histogram of its middle sixteenth of slices are computed
(tsallis_histogram), and both are labelled with the exhaustive search's
threshold of the whole volume (tsallis_search); the volume itself is not
kept. The target is the uniform distribution over the thresholds that give
the labelled partition (the labelled level and the empty levels after it).

Training: Adam on the mean soft-target cross-entropy (the library's
forward, backward and optimiser kernels), minibatches drawn with a seeded
generator. The result is written with tsallis_proposer_save. With
--checkpoint the training state is saved every --checkpoint-every steps and
--resume continues an interrupted run exactly.

    python -m paper_2012_10684_gb300.proposer --out weights.bin
    python -m paper_2012_10684_gb300.proposer --two-d --volumes 300 --steps 6000 --batch 256 --out w2d.bin
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np
import torch

import paper_2012_10684_gb300 as tg


def soft_targets(hist: torch.Tensor, t: torch.Tensor) -> torch.Tensor:
    """y [n][4096]: uniform over [t, e) where e is the first non-empty level
    after t (rows with t = -1 stay zero)."""
    n = hist.shape[0]
    idx = torch.arange(4096, device=hist.device).expand(n, 4096)
    tt = t.to(torch.int64).view(-1, 1)
    after = (hist > 0) & (idx > tt)
    e = torch.where(after, idx, torch.full_like(idx, 4095)).min(dim=1, keepdim=True).values
    y = ((idx >= tt) & (idx < e) & (tt >= 0)).to(torch.float32)
    s = y.sum(dim=1, keepdim=True)
    return y / torch.where(s > 0, s, torch.ones_like(s))


def make_dataset(n: int, seed: int, dmin: int, dmax: int, q: float = 0.8, nx: int = 512, ny: int = 512,
                 device="cuda", log_every: int = 0):
    """(hist [n][4096], sub [n][4096], t [n], status [n]) from n generated
    volumes: each volume's histogram, the histogram of the middle sixteenth
    of its slices (what a batch's first-pass prediction reads), and the
    exhaustive search's threshold of the whole volume."""
    import phantom
    rng = np.random.default_rng(seed)
    p = tg.tsallis_params(q=q, mode="volume")
    hist = torch.empty((n, 4096), dtype=torch.int32, device=device)
    sub = torch.empty((n, 4096), dtype=torch.int32, device=device)
    buf = torch.empty(dmax * ny * nx, dtype=torch.int16, device=device)
    t0 = time.time()
    for i in range(n):
        nz = int(rng.integers(dmin, dmax + 1))
        spec = phantom.chest_volume(seed * 100000 + i, nx, ny, nz, generations=int(rng.integers(4, 9)),
                                    noise_sd=int(rng.integers(5, 31)), vol_id=i)
        vol = buf[: nz * ny * nx].view(nz, ny, nx)
        phantom.generate_cuda(spec, out=vol)
        tg.tsallis_histogram(vol, p, hist[i:i + 1])
        ns = max(1, nz // 16)
        z0 = (nz - ns) // 2
        tg.tsallis_histogram(vol[z0:z0 + ns], p, sub[i:i + 1])
        if log_every and (i + 1) % log_every == 0:
            print("generated %d volumes, %.1f s" % (i + 1, time.time() - t0), flush=True)
    t, _, st = tg.tsallis_search(hist, p)
    return hist, sub, t, st


def make_dataset2d(nvol: int, seed: int, nz: int = 24, q: float = 0.8, nx: int = 512, ny: int = 512,
                   device="cuda", log_every: int = 0):
    """(hist [n][256][256], t [n][2], status [n]) for the 2-D search's
    proposer: from each of nvol generated chest volumes of nz slices, the
    2-D histogram (256 grey x 256 mean levels) of every slice (3x3 window)
    and of the volume (3x3x3 window), labelled with the exhaustive 2-D
    search's pair."""
    import phantom
    rng = np.random.default_rng(seed)
    ps = tg.tsallis_params(q=q, mode="slice", two_d=True)
    pv = tg.tsallis_params(q=q, mode="volume", two_d=True)
    per = nz + 1
    hist = torch.empty((nvol * per, 256, 256), dtype=torch.int32, device=device)
    buf = torch.empty(nz * ny * nx, dtype=torch.int16, device=device)
    t0 = time.time()
    for i in range(nvol):
        spec = phantom.chest_volume(seed * 100000 + i, nx, ny, nz, generations=int(rng.integers(4, 9)),
                                    noise_sd=int(rng.integers(5, 31)), vol_id=i)
        vol = buf.view(nz, ny, nx)
        phantom.generate_cuda(spec, out=vol)
        tg.tsallis_histogram(vol, ps, hist[i * per: i * per + nz])
        tg.tsallis_histogram(vol, pv, hist[i * per + nz: (i + 1) * per])
        if log_every and (i + 1) % log_every == 0:
            print("generated %d volumes, %.1f s" % (i + 1, time.time() - t0), flush=True)
    t, _, st = tg.tsallis_search(hist, ps)
    return hist, t, st


def cell_targets(t: torch.Tensor) -> torch.Tensor:
    """y [n][4096]: one-hot on the cell 64 * (t // 4) + s // 4 of each pair
    (rows without a pair stay zero)."""
    n = t.shape[0]
    y = torch.zeros((n, 4096), dtype=torch.float32, device=t.device)
    ok = t[:, 0] >= 0
    cell = (t[:, 0].long() // 4) * 64 + t[:, 1].long() // 4
    y[torch.nonzero(ok).squeeze(1), cell[ok]] = 1.0
    return y


def _pack_state(s: int, gen: torch.Generator) -> bytes:
    """The trainer's own state stored in a checkpoint: the next step number
    and the minibatch generator's state."""
    return int(s).to_bytes(8, "little") + gen.get_state().cpu().numpy().tobytes()


def train(x: torch.Tensor, y: torch.Tensor, steps: int, batch: int, lr: float, seed: int, init_seed: int = 1,
          log_every: int = 0, checkpoint: str | None = None, checkpoint_every: int = 0, resume: str | None = None,
          stop_after: int | None = None):
    """Trains the context's proposer from a seeded initialisation; returns
    the loss of every step taken (NaN for the steps a resumed run skipped).

    With checkpoint and checkpoint_every, the parameters, Adam moments and
    step count (tsallis_proposer_checkpoint_save) and the minibatch
    generator's state are written every checkpoint_every steps; resume
    restores them and continues, so that a resumed run ends with the same
    parameters, bit for bit, as one that was never interrupted. stop_after
    ends the run after that many steps (an interrupted run)."""
    gen = torch.Generator(device=x.device)
    gen.manual_seed(seed)
    start = 0
    if resume:
        user = tg.proposer_checkpoint_load(resume, device=x.device)
        start = int.from_bytes(user[:8], "little")
        gen.set_state(torch.frombuffer(bytearray(user[8:]), dtype=torch.uint8))
    else:
        g = np.random.default_rng(init_seed)
        params = []
        for fan_out, fan_in in ((256, 256), (256, 256), (4096, 256)):
            bound = math.sqrt(6.0 / (fan_in + fan_out))
            params.append(g.uniform(-bound, bound, fan_out * fan_in))
            params.append(np.zeros(fan_out))
        tg.proposer_set(np.concatenate(params).astype(np.float32), x.device)
    losses = torch.full((steps,), float("nan"), dtype=torch.float32, device=x.device)
    n = x.shape[0]
    end = steps if stop_after is None else min(steps, stop_after)
    for s in range(start, end):
        # cosine decay of the learning rate
        lr_s = lr * 0.5 * (1 + math.cos(math.pi * s / steps))
        idx = torch.randint(0, n, (batch,), device=x.device, generator=gen)
        loss, _ = tg.proposer_train_step(x[idx], y[idx], lr_s)
        losses[s] = loss[0]
        if log_every and (s + 1) % log_every == 0:
            print("step %d loss %.4f" % (s + 1, float(losses[s])), flush=True)
        if checkpoint and checkpoint_every and (s + 1) % checkpoint_every == 0:
            tg.proposer_checkpoint_save(checkpoint, _pack_state(s + 1, gen), device=x.device)
    return losses.cpu().numpy()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--volumes", type=int, default=20000)
    ap.add_argument("--dmin", type=int, default=120)
    ap.add_argument("--dmax", type=int, default=600)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=2012106845)
    ap.add_argument("--out", required=True)
    ap.add_argument("--checkpoint", help="training checkpoint written every --checkpoint-every steps")
    ap.add_argument("--checkpoint-every", type=int, default=1000)
    ap.add_argument("--resume", help="checkpoint to continue from (same data arguments)")
    ap.add_argument("--two-d", action="store_true",
                    help="train the 2-D search's proposer (slot 1) on per-slice and per-volume 2-D histograms")
    ap.add_argument("--nz", type=int, default=24, help="slices per generated volume (2-D training)")
    args = ap.parse_args()
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    t0 = time.time()
    if args.two_d:
        tg.proposer_select(1)
        hist, t, st = make_dataset2d(args.volumes, args.seed, nz=args.nz, log_every=50)
        x = tg.proposer_features(hist)
        y = cell_targets(t)
        del hist
        torch.cuda.synchronize()
        t1 = time.time()
        losses = train(x, y, args.steps, args.batch, args.lr, args.seed, log_every=500,
                       checkpoint=args.checkpoint, checkpoint_every=args.checkpoint_every, resume=args.resume)
        torch.cuda.synchronize()
        tg.proposer_save(args.out)
        print("2-D: %d histograms, data %.1f s, training %.1f s, final loss %.4f" % (
            x.shape[0], t1 - t0, time.time() - t1, np.nanmean(losses[-100:])))
        return
    hist, sub, t, st = make_dataset(args.volumes, args.seed, args.dmin, args.dmax, log_every=1000)
    assert bool(((st & 0xff) == 0).all())
    # each volume gives two examples with the same target: its histogram
    # (for the window search) and its middle sixteenth (for the prediction)
    x = torch.cat([tg.proposer_features(hist), tg.proposer_features(sub)])
    y = soft_targets(hist, t)
    y = torch.cat([y, y])
    torch.cuda.synchronize()
    t1 = time.time()
    losses = train(x, y, args.steps, args.batch, args.lr, args.seed, log_every=500, checkpoint=args.checkpoint,
                   checkpoint_every=args.checkpoint_every, resume=args.resume)
    torch.cuda.synchronize()
    tg.proposer_save(args.out)
    print("data %.1f s, training %.1f s, final loss %.4f" % (t1 - t0, time.time() - t1,
                                                             np.nanmean(losses[-100:])))


if __name__ == "__main__":
    main()
