"""End-to-end neurosymbolic training through the differentiable fixpoint (a
synthetic Pathfinder-like task): the CNN's edge probabilities feed a batched
reachability fixpoint, whose target tags are trained with binary
cross-entropy through lob_backward."""
import numpy as np
import pytest

from paper_2503_21937_gb300 import pathfinder as PF

pytestmark = pytest.mark.gpu


def test_batches_are_seeded_and_balanced():
    a = PF.make_batch(6, 16, seed=3)
    b = PF.make_batch(6, 16, seed=3)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert 0.25 <= a[3].mean() <= 0.75  # both labels present


def test_forward_matches_oracle_on_the_predicted_probabilities():
    """The target tags the training step consumes equal the oracle's
    diff-max-min reach tags on the same edge probabilities."""
    import torch
    from tests.common import oracle_run
    torch.manual_seed(0)
    model = PF.build_model().cuda()
    side, batch = 5, 4
    pf = PF.Pathfinder(side, batch)
    img, st, tg, lab = PF.make_batch(side, batch, seed=11)
    with torch.no_grad():
        logits = model(torch.from_numpy(img).cuda())[:, 0].flatten(1)
        p = torch.sigmoid(logits[:, pf.pix]).cpu().numpy()
    pred = pf.forward(model, torch.from_numpy(img).cuda(), torch.from_numpy(st).cuda(),
                      torch.from_numpy(tg).cuda()).detach().cpu().numpy()
    u, v, _, _ = PF.grid_edges(side)
    for i in range(batch):
        src = np.concatenate([u, v]).astype(np.uint32)
        dst = np.concatenate([v, u]).astype(np.uint32)
        probs = np.concatenate([p[i], p[i]]).astype(np.float32)
        res = oracle_run(PF.PROGRAM, {"edge": ((src, dst), probs), "start": ((np.array([st[i]], np.uint32),),)},
                         "diff_max_min")
        rel = res.relation("reach")
        k = int(np.searchsorted(rel.cols[0], tg[i]))
        assert rel.cols[0][k] == tg[i]
        assert np.float32(rel.tags[k]) == np.float32(pred[i])


def test_training_reduces_the_loss():
    out = PF.train(side=6, batch=32, steps=60, seed=1)
    loss = np.array([h[0] for h in out["history"]])
    acc = np.array([h[1] for h in out["history"]])
    assert loss[-10:].mean() < 0.7 * loss[:10].mean()
    assert acc[-10:].mean() > 0.8
