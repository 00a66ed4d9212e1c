"""End-to-end neurosymbolic training on a synthetic Pathfinder-like task (the
paper's Sec. 2 example: a neural network predicts, from an image, the
probability of every edge of an n x n grid; a Datalog program decides whether
two marked dots are connected; the loss on that decision trains the network
through the differentiable fixpoint).

Each sample is an image of side 2n - 1 over the grid: node pixels at even
coordinates, the pixel between two neighbouring nodes lit when the edge
between them is drawn, plus noise; a second channel marks the two dots.  Half
the samples draw a random path between the dots (connected), half draw paths
that keep them in different components (not connected); distractor segments
are added to both.  The network is a small CNN whose per-pixel logit at an
edge's midpoint is that edge's probability.  The program

    reach(x) :- start(x).
    reach(y) :- reach(x), edge(x, y).

runs over all samples in one engine run (a sample id per fact), with
diff-max-min tags: the tag of reach(target) is the strength of the strongest
path, and the binary cross-entropy of that tag against the label is
back-propagated through lob_backward into the CNN.

The generators are seeded (SplitMix64 streams of ``workloads``) and hold none
of the method's arithmetic; everything the fixpoint computes runs in the
engine's CUDA kernels.
"""
from __future__ import annotations

import time

import numpy as np

from . import workloads as W

PROGRAM = W.REACH_PROGRAM


def grid_edges(side: int):
    """Undirected edges of the side x side grid: (u, v) node pairs and the
    image pixel (row, col) at each edge's midpoint."""
    u, v, pr, pc = [], [], [], []
    for r in range(side):
        for c in range(side):
            a = r * side + c
            if c + 1 < side:
                u.append(a); v.append(a + 1); pr.append(2 * r); pc.append(2 * c + 1)
            if r + 1 < side:
                u.append(a); v.append(a + side); pr.append(2 * r + 1); pc.append(2 * c)
    return (np.array(u, np.int64), np.array(v, np.int64), np.array(pr, np.int64), np.array(pc, np.int64))


def _components(side, u, v, drawn):
    parent = list(range(side * side))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b, d in zip(u.tolist(), v.tolist(), drawn.tolist()):
        if d:
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[ra] = rb
    return [find(x) for x in range(side * side)]


def _random_path(s: W.Stream, side, start, length):
    """A self-avoiding random walk of up to `length` steps from `start`."""
    path = [start]
    seen = {start}
    for _ in range(length):
        r, c = divmod(path[-1], side)
        nbr = [(r + dr) * side + (c + dc) for dr, dc in ((0, 1), (1, 0), (0, -1), (-1, 0))
               if 0 <= r + dr < side and 0 <= c + dc < side and (r + dr) * side + (c + dc) not in seen]
        if not nbr:
            break
        nxt = nbr[int(s.below(1, len(nbr))[0])]
        path.append(nxt)
        seen.add(nxt)
    return path


def make_batch(side: int, batch: int, seed: int, noise: float = 0.15):
    """Seeded batch: images (batch, 2, 2*side-1, 2*side-1) float32, start and
    target node per sample, labels (1 connected, 0 not)."""
    s = W.stream(900_000 + seed)
    u, v, pr, pc = grid_edges(side)
    eid = {}
    for k, (a, b) in enumerate(zip(u.tolist(), v.tolist())):
        eid[(a, b)] = k
        eid[(b, a)] = k
    hw = 2 * side - 1
    images = np.zeros((batch, 2, hw, hw), np.float32)
    starts = np.zeros(batch, np.int64)
    targets = np.zeros(batch, np.int64)
    labels = np.zeros(batch, np.float32)
    for i in range(batch):
        want = i % 2 == 0
        for _attempt in range(100):
            drawn = np.zeros(len(u), bool)
            a = int(s.below(1, side * side)[0])
            path = _random_path(s, side, a, 2 * side)
            for x, y in zip(path[:-1], path[1:]):
                drawn[eid[(x, y)]] = True
            for _ in range(side // 2):  # distractor segments
                seg = _random_path(s, side, int(s.below(1, side * side)[0]), side // 2)
                for x, y in zip(seg[:-1], seg[1:]):
                    drawn[eid[(x, y)]] = True
            comp = _components(side, u, v, drawn)
            if want:
                b = path[-1]
                if b == a:
                    continue
            else:
                others = [x for x in range(side * side) if comp[x] != comp[a]]
                if not others:
                    continue
                b = others[int(s.below(1, len(others))[0])]
            break
        starts[i], targets[i] = a, b
        labels[i] = float(comp[a] == comp[b])
        img = images[i, 0]
        img[0::2, 0::2] = 0.5
        img[pr[drawn], pc[drawn]] = 1.0
        ra, ca = divmod(a, side)
        rb, cb = divmod(b, side)
        images[i, 1, 2 * ra, 2 * ca] = 1.0
        images[i, 1, 2 * rb, 2 * cb] = 1.0
    images[:, 0] += noise * s.normal(images[:, 0].size).reshape(images[:, 0].shape).astype(np.float32)
    return images, starts, targets, labels


def build_model(channels: int = 32):
    """Per-pixel edge logits from the two-channel image (fully convolutional)."""
    import torch.nn as nn
    return nn.Sequential(
        nn.Conv2d(2, channels, 3, padding=1), nn.ReLU(),
        nn.Conv2d(channels, channels, 3, padding=1), nn.ReLU(),
        nn.Conv2d(channels, channels, 3, padding=1), nn.ReLU(),
        nn.Conv2d(channels, 1, 1))


class Pathfinder:
    """One (side, batch) configuration: the grid's edge list on the device and
    the forward pass image -> edge probabilities -> fixpoint -> target tags."""

    def __init__(self, side: int, batch: int, semiring: str = "diff_max_min", device: str = "cuda"):
        import torch
        self.side, self.batch, self.semiring, self.device = side, batch, semiring, device
        u, v, pr, pc = grid_edges(side)
        self.n_edges = len(u)
        self.pix = torch.from_numpy(pr * (2 * side - 1) + pc).to(device)
        # both directions of every edge, for every sample (sample-major)
        src = np.concatenate([u, v])
        dst = np.concatenate([v, u])
        sid = np.repeat(np.arange(batch), 2 * len(u))
        self.cols = torch.from_numpy(np.stack([np.tile(src, batch), np.tile(dst, batch)]).astype(np.int32)).to(device)
        self.sids = torch.from_numpy(sid.astype(np.int32)).to(device)

    def forward(self, model, images, starts, targets):
        """Connectivity probability of each sample (differentiable)."""
        import torch
        from .autograd import fixpoint
        logits = model(images)[:, 0].flatten(1)           # (batch, pixels)
        p = torch.sigmoid(logits[:, self.pix])            # (batch, n_edges)
        probs = torch.cat([p, p], dim=1).reshape(-1)      # both directions, sample-major
        start = starts.to(torch.int32).reshape(1, -1)      # start(x): one row per sample
        out = fixpoint(PROGRAM, {"edge": (self.cols, probs, self.sids),
                                 "start": (start, None, torch.arange(self.batch, dtype=torch.int32,
                                                                     device=self.device))},
                       self.semiring, outputs=["reach"])
        rc, rt, rs = out["reach"]
        key = rs.to(torch.int64) * (self.side * self.side) + rc[0].to(torch.int64)
        want = torch.arange(self.batch, device=self.device, dtype=torch.int64) * (self.side * self.side) + targets
        idx = torch.searchsorted(key, want)
        return rt[idx.clamp(max=key.numel() - 1)]


def train(side: int = 6, batch: int = 32, steps: int = 60, lr: float = 3e-3, semiring: str = "diff_max_min",
          seed: int = 0, log_every: int = 10):
    """Train the CNN for `steps` steps on fresh seeded batches; returns the
    loss / accuracy history and the time per step."""
    import torch
    torch.manual_seed(seed)
    model = build_model().cuda()
    opt = torch.optim.Adam(model.parameters(), lr=lr)
    pf = Pathfinder(side, batch, semiring)
    hist = []
    t_total = 0.0
    for step in range(steps):
        img, st, tg, lab = make_batch(side, batch, seed * 100_000 + step)
        img = torch.from_numpy(img).cuda()
        st, tg, lab = (torch.from_numpy(st).cuda(), torch.from_numpy(tg).cuda(), torch.from_numpy(lab).cuda())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pred = pf.forward(model, img, st, tg).clamp(1e-6, 1 - 1e-6)
        loss = torch.nn.functional.binary_cross_entropy(pred, lab)
        opt.zero_grad()
        loss.backward()
        opt.step()
        torch.cuda.synchronize()
        t_total += time.perf_counter() - t0
        acc = float(((pred > 0.5).float() == lab).float().mean())
        hist.append((float(loss.detach()), acc))
    return {"history": hist, "s_per_step": t_total / steps}


def sweep(sides=(8, 16, 32), batch: int = 64, steps: int = 5, semiring: str = "diff_max_min"):
    """Training-step throughput (forward + backward + optimizer step, samples
    per second) over grid sides (the shape of the paper's grid-size scaling
    study); the first step of each side is an untimed warm-up."""
    import torch
    out = {}
    for side in sides:
        torch.manual_seed(0)
        model = build_model().cuda()
        opt = torch.optim.Adam(model.parameters(), lr=1e-3)
        pf = Pathfinder(side, batch, semiring)
        batches = [make_batch(side, batch, 7_000 + side * 100 + k) for k in range(steps + 1)]
        times = []
        for k, (img, st, tg, lab) in enumerate(batches):
            img = torch.from_numpy(img).cuda()
            st, tg, lab = (torch.from_numpy(st).cuda(), torch.from_numpy(tg).cuda(), torch.from_numpy(lab).cuda())
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pred = pf.forward(model, img, st, tg).clamp(1e-6, 1 - 1e-6)
            loss = torch.nn.functional.binary_cross_entropy(pred, lab)
            opt.zero_grad()
            loss.backward()
            opt.step()
            torch.cuda.synchronize()
            if k:
                times.append(time.perf_counter() - t0)
        ms = 1e3 * float(np.median(times))
        out[str(side)] = {"batch": batch, "ms_per_step": round(ms, 2), "samples_per_s": round(batch / (ms / 1e3), 1)}
    return out
