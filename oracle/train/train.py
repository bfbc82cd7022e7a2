"""Train the NENO6 classifier (Sec. 3.3, Table 2) and write the weights file.

Training infrastructure (oracle side): the product library only reads the
resulting file.  Binary cross entropy of Eq. (Crossentropy) on the sigmoid
outputs (computed from the logits), Adam, mini-batch m = 175, learning rate
1e-4 halved at epochs 40, 90, 160, 300 and 700, the training set reshuffled
every epoch; 6-64-32-16-8-4 with ReLU (Sec. 3.1).  Plain PyTorch on the CPU,
float32 arithmetic; the weights are stored as float64.

    python -m oracle.train.train --epochs 1000 --out weights/neno6_mlp_6x64x32x16x8x4.bin

The weights file is rewritten after every epoch (atomic rename), and one line
per epoch (train/validation BCE, validation F1) is appended to --log.
"""
import argparse
import os
import time

import numpy as np
import torch

from ..weights import Net
from . import datagen

MILESTONES = (40, 90, 160, 300, 700)


def make_model(widths=(6, 64, 32, 16, 8, 4)):
    layers = []
    for i, (a, b) in enumerate(zip(widths[:-1], widths[1:])):
        layers.append(torch.nn.Linear(a, b))
        if i < len(widths) - 2:
            layers.append(torch.nn.ReLU())
    return torch.nn.Sequential(*layers)


def to_net(model):
    lin = [m for m in model if isinstance(m, torch.nn.Linear)]
    return Net([(m.weight.detach().double().numpy(), m.bias.detach().double().numpy()) for m in lin])


def f1_scores(logits, y):
    """Eq. (F1score) for each class convention: positive = discarded (eta=1)
    and positive = kept (eta=0)."""
    pred = logits > 0
    yt = y.astype(bool)
    out = {}
    for name, p, t in (("rough", pred, yt), ("smooth", ~pred, ~yt)):
        tp = np.sum(p & t)
        fp = np.sum(p & ~t)
        fn = np.sum(~p & t)
        out[name] = 2 * tp / max(2 * tp + fp + fn, 1)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--epochs", type=int, default=1000)
    ap.add_argument("--samples", type=int, default=709000)
    ap.add_argument("--batch", type=int, default=175)
    ap.add_argument("--lr", type=float, default=1e-4)
    ap.add_argument("--seed", type=int, default=20220717)
    ap.add_argument("--threads", type=int, default=2)
    ap.add_argument("--widths", default="6,64,32,16,8,4",
                    help="layer widths, inputs first (Sec. 3.1: 6,64,32,16,8,4)")
    ap.add_argument("--out", default="weights/neno6_mlp_6x64x32x16x8x4.bin")
    ap.add_argument("--log", default="weights/train_log.txt")
    args = ap.parse_args()
    torch.set_num_threads(args.threads)
    torch.manual_seed(args.seed)
    (Xtr, ytr), (Xva, yva), _ = datagen.dataset(args.samples, args.seed)
    Xtr_t = torch.from_numpy(Xtr.astype(np.float32))
    ytr_t = torch.from_numpy(ytr.astype(np.float32))
    Xva_t = torch.from_numpy(Xva.astype(np.float32))
    yva_t = torch.from_numpy(yva.astype(np.float32))
    model = make_model(tuple(int(w) for w in args.widths.split(",")))
    opt = torch.optim.Adam(model.parameters(), lr=args.lr)
    sched = torch.optim.lr_scheduler.MultiStepLR(opt, milestones=list(MILESTONES), gamma=0.5)
    bce = torch.nn.BCEWithLogitsLoss()  # mean over outputs and batch = Eq. (Crossentropy)
    gen = torch.Generator().manual_seed(args.seed)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    with open(args.log, "a") as lf:
        lf.write("# samples %d (train %d, val %d), batch %d, lr %g, milestones %s, widths %s\n"
                 % (args.samples, len(Xtr), len(Xva), args.batch, args.lr, MILESTONES, args.widths))
    for ep in range(1, args.epochs + 1):
        t0 = time.time()
        model.train()
        perm = torch.randperm(len(Xtr_t), generator=gen)
        tot, nb = 0.0, 0
        for s in range(0, len(perm), args.batch):
            idx = perm[s:s + args.batch]
            opt.zero_grad(set_to_none=True)
            loss = bce(model(Xtr_t[idx]), ytr_t[idx])
            loss.backward()
            opt.step()
            tot += loss.item()
            nb += 1
        sched.step()
        model.eval()
        with torch.no_grad():
            lv = model(Xva_t)
            vloss = bce(lv, yva_t).item()
        f1 = f1_scores(lv.numpy(), yva)
        net = to_net(model)
        tmp = args.out + ".tmp"
        net.save(tmp)
        os.replace(tmp, args.out)
        line = ("epoch %4d  train_bce %.5f  val_bce %.5f  val_F1_rough %.4f  val_F1_smooth %.4f"
                "  lr %.2e  %.1fs" % (ep, tot / nb, vloss, f1["rough"], f1["smooth"],
                                      opt.param_groups[0]["lr"], time.time() - t0))
        print(line, flush=True)
        with open(args.log, "a") as lf:
            lf.write(line + "\n")


if __name__ == "__main__":
    main()
