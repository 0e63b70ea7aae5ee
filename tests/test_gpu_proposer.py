"""The learned radius proposer end to end on the GPU (not in the paper: it
grows every sphere by sphere shrinking from a radius above the shape,
Sec. 5.1).

* rpd_pin_features must match the oracle's restatement of the features.
* rpd_shrink_warm must reach the plain method's sphere from any proposal:
  from above it, in no more iterations; from below it, by starting over.
* A network trained by the library's own kernels on (pin features ->
  log2 of the shrunk radius) pairs of seeded training shapes must, on a
  held-out shape, leave the repair loops' result unchanged (same spheres,
  same failing counts: the shrinking and the exact RPD check decide) while
  cutting the shrinking iterations.
"""
import numpy as np
import pytest
import torch

from oracle import mlp as ref
from paper_2403_18761_gb300 import build_workload, Mlp
from rpd_inputs import genus_slab

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _box(w):
    q, _, _ = w.ints()
    v = q * (1.0 / float(1 << w.grid_bits))
    return v.min(axis=0), v.max(axis=0)


def test_features_match_oracle():
    w = genus_slab(2, h=0.15, ns=64)
    ctx = build_workload(w)
    P, N, F = ctx.rpd_surface_samples()
    _, r, _ = ctx.rpd_shrink(P, N, F)
    x, t = ctx.rpd_pin_features(P, N, r)
    lo, hi = _box(w)
    want = ref.pin_features(P.cpu().numpy(), N.cpu().numpy(), lo, hi)
    assert np.abs(x.cpu().numpy() - want).max() <= 2e-5
    wt = ref.radius_target(r.cpu().numpy(), lo, hi)
    assert np.abs(t.cpu().numpy() - wt).max() <= 2e-5


def test_warm_start_reaches_the_plain_sphere():
    w = genus_slab(1, h=0.15, ns=64)
    ctx = build_workload(w)
    P, N, F = ctx.rpd_surface_samples()
    sel = torch.arange(0, P.shape[0], 5, device=P.device)
    P, N, F = P[sel].contiguous(), N[sel].contiguous(), F[sel].contiguous()
    c0, r0, it0 = ctx.rpd_shrink(P, N, F)
    ok = it0 < 99
    assert ok.float().mean() > 0.99
    # from above: the same sphere, never more iterations
    c1, r1, it1, rs1 = ctx.rpd_shrink_warm(P, N, F, 1.25 * r0)
    assert torch.all(rs1 == 0)
    assert torch.all(torch.abs(r1 - r0)[ok] <= 1e-9 * r0[ok])
    assert torch.all((it1 <= it0)[ok])
    assert it1.sum() < it0.sum()
    # from below: every proposal rejected, then exactly the plain path
    c2, r2, it2, rs2 = ctx.rpd_shrink_warm(P, N, F, 0.5 * r0)
    assert torch.all(rs2 == 1)
    assert torch.equal(r2[ok], r0[ok]) and torch.equal(c2[ok], c0[ok])
    assert torch.equal(it2[ok], it0[ok] + 1)
    # zero proposals are the plain start
    _, r3, it3, rs3 = ctx.rpd_shrink_warm(P, N, F, torch.zeros_like(r0))
    assert torch.equal(r3, r0) and torch.equal(it3, it0) and torch.all(rs3 == 0)


def _training_pairs(shapes):
    xs, ts = [], []
    for w in shapes:
        ctx = build_workload(w)
        P, N, F = ctx.rpd_surface_samples()
        _, r, it = ctx.rpd_shrink(P, N, F)
        x, t = ctx.rpd_pin_features(P, N, r)
        keep = torch.isfinite(t)
        xs.append(x[keep])
        ts.append(t[keep])
    return torch.cat(xs), torch.cat(ts)


def test_learned_proposer_keeps_the_result_and_saves_shrinking():
    # training shapes: genus 0, 1, 2, 4, 5 (two seeds each); held out: genus 3
    shapes = [genus_slab(g, seed=s, h=0.075, ns=64) for g in (0, 1, 2, 4, 5) for s in (11, 12)]
    x, t = _training_pairs(shapes)
    assert x.shape[0] >= 50_000
    g = torch.Generator(device="cpu").manual_seed(0)
    perm = torch.randperm(x.shape[0], generator=g).to(x.device)
    x, t = x[perm].contiguous(), t[perm].contiguous()
    net = Mlp(seed=7)
    _, l0 = net.grad(x, t)
    net.train(x, t, steps=3000, batch=1024, lr=1e-3)
    _, l1 = net.grad(x, t)
    assert l1 < 0.25 * l0, (l0, l1)

    held = genus_slab(3, seed=13, h=0.075, ns=64)
    res = {}
    for mode in ("plain", "learned"):
        ctx = build_workload(held)
        if mode == "learned":
            ctx.rpd_set_proposer(net, 1.25)
        rep = ctx.rpd_repair_geometry(0.02, 48)
        c, r = ctx.rpd_spheres()
        res[mode] = (rep, c.cpu().numpy(), r.cpu().numpy(), ctx.rpd_shrink_counters())
    (rp, cp, rp_, kp), (rl, cl, rl_, kl) = res["plain"], res["learned"]
    print("plain", rp, kp, "learned", rl, kl)
    assert rp == rl
    assert np.array_equal(cp, cl) and np.array_equal(rp_, rl_)
    assert kp[0] == kl[0] and kp[0] > 0
    assert kl[1] < kp[1], (kp, kl)
