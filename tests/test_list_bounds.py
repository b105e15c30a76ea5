"""The candidate lists' skip rule, restated in float32 numpy and checked on adversarial inputs (CPU).

The ICP kernel keeps, per source point, up to 8 targets sorted by distance from the position p_b where the
list was built, with 8-bit codes c_k such that c_k * sigma / 127.5 is a lower bound on
|q_k - p_b| - |q_0 - p_b|.  At a later position p it does not load entry k when that bound exceeds
2 |p - p_b| plus a relative margin: the argument (triangle inequality, then float32 rounding) says such an
entry's float32 d2 at p is strictly above entry 0's, so it can neither win nor tie.  This test restates the
kernel's float32 formulas (every operation rounded on its own, square roots perturbed by up to +-4e-7 of
their value, more than the hardware reciprocal square root's error) and checks that claim on random and
near-tied configurations, including targets on a lattice with equal distances, and on collinear
configurations where the triangle inequality is tight (entry 0 behind the motion, entry k ahead, the gap a
hair either side of twice the motion).  Codes rounded up instead of down make it fail.
"""
from __future__ import annotations

import numpy as np

f32 = np.float32
GAP_SCALE = f32(127.5)
INV_GAP_SCALE = f32(1.0) / f32(127.5)


def fast_sqrt(x, g):
    """sqrt of max(x, 1e-30) in float32 with a relative error of up to 4e-7 either way."""
    y = np.maximum(x, f32(1e-30)).astype(f32)
    s = np.sqrt(y).astype(f32)
    eps = g.uniform(-4e-7, 4e-7, size=s.shape).astype(np.float64)
    return (s.astype(np.float64) * (1.0 + eps)).astype(f32)


def dist2_rn(p, q):
    d = (p - q).astype(f32)
    return ((d[..., 0] * d[..., 0]).astype(f32) + (d[..., 1] * d[..., 1]).astype(f32)).astype(f32) + \
        (d[..., 2] * d[..., 2]).astype(f32)


def codes(d2, sigma, g, round_up=False):
    """Gap codes of entries 1.. from the sorted float32 d2 of the entries at p_b (as the list store forms them;
    round_up plants the mistake of codes rounded up from the plain distance difference)."""
    if round_up:
        gk = (np.sqrt(d2).astype(f32) - np.sqrt(d2[:, :1]).astype(f32)).astype(f32)
        c = np.ceil((gk * (GAP_SCALE / sigma).astype(f32)).astype(f32))
    else:
        r0 = fast_sqrt((d2[:, :1] * f32(1.0002)).astype(f32), g)
        inv = (GAP_SCALE / sigma).astype(f32)
        gk = (fast_sqrt((d2 * f32(0.9998)).astype(f32), g) - r0).astype(f32)
        c = ((gk * inv).astype(f32) * f32(0.9999)).astype(f32)
    code = np.where(c > 0, np.minimum(np.floor(np.minimum(c, f32(1e9))), 255.0), 0.0).astype(np.uint32)
    code[:, 0] = 0
    return code


def skipped(p, pb, rho2, code, sigma, g):
    moved = dist2_rn(p, pb)
    dm = fast_sqrt((moved * f32(1.0001)).astype(f32), g)
    rr = fast_sqrt((rho2 * f32(1.0001)).astype(f32), g)
    rel = (f32(2e-4) * (rr + dm).astype(f32)).astype(f32)
    thr = (((f32(2.0) * dm).astype(f32) + rel).astype(f32) * f32(1.0001)).astype(f32)
    unit = (sigma * INV_GAP_SCALE).astype(f32)
    lb = (code.astype(f32) * unit).astype(f32)
    skip = lb > thr[:, None]
    skip[:, 0] = False
    return skip


def violations(pb, q, p, sigma, g, round_up=False):
    """Entries the rule skips whose float32 d2 at p is not strictly above entry 0's."""
    d2b = dist2_rn(pb[:, None, :], q)
    order = np.lexsort((np.arange(q.shape[1])[None, :].repeat(len(q), 0), d2b), axis=1)
    q = np.take_along_axis(q, order[:, :, None], axis=1)
    d2b = np.take_along_axis(d2b, order, axis=1)
    rho2 = (d2b.max(axis=1) * f32(1.0001)).astype(f32)
    code = codes(d2b, sigma, g, round_up)
    skip = skipped(p, pb, rho2, code, sigma, g)
    d2p = dist2_rn(p[:, None, :], q)
    bad = skip & ~(d2p > d2p[:, :1])
    return int(bad.sum()), int(skip.sum())


def _configs(g, n, spread, motion, lattice=None):
    pb = g.uniform(-4.0, 4.0, (n, 3)).astype(f32)
    if lattice:
        pb = (np.round(pb / lattice) * lattice).astype(f32)
        off = g.integers(-3, 4, (n, 8, 3)) * lattice
        q = (pb[:, None, :] + off).astype(f32)
    else:
        q = (pb[:, None, :] + g.normal(0.0, spread, (n, 8, 3))).astype(f32)
    dirs = g.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    p = (pb + dirs * g.uniform(0.0, motion, (n, 1))).astype(f32)
    return pb, q, p


def _collinear(g, n, sigma):
    """Entry 0 at distance a behind the motion u, entry 1 ahead at a + G, the point moved by delta along u:
    at p entry 1 is nearer exactly when G < 2 delta.  G sits within 0.5 % of 2 delta either side."""
    pb = g.uniform(-2.0, 2.0, (n, 3)).astype(f32)
    u = g.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    a = g.uniform(0.002, 0.008, (n, 1))
    delta = g.uniform(0.05, 0.5, (n, 1)) * float(sigma)
    G = 2.0 * delta * (1.0 + g.uniform(-0.005, 0.005, (n, 1)))
    q0 = pb - u * a
    q1 = pb + u * (a + G)
    # the other entries further ahead, all within the list's reach of d0 + sigma
    far = q1[:, None, :] + u[:, None, :] * (np.arange(1, 7)[None, :, None] * 0.1 * float(sigma))
    q = np.concatenate([q0[:, None, :], q1[:, None, :], far], axis=1).astype(f32)
    p = (pb + u * delta).astype(f32)
    return pb, q, p


def test_skip_rule_never_drops_a_winner_or_a_tie():
    g = np.random.default_rng(7)
    sigma = f32(0.002)
    total_skips = 0
    for spread, motion, lattice in ((0.003, 0.0005, None), (0.003, 0.002, None), (0.0002, 1e-5, None),
                                    (0.01, 0.004, None), (0.003, 0.0, None), (None, 0.0, 0.001),
                                    (None, 1e-4, 0.001), (None, 0.0, 0.0005)):
        pb, q, p = _configs(g, 20000, spread or 0.0, motion, lattice)
        bad, skips = violations(pb, q, p, sigma, g)
        assert bad == 0, (spread, motion, lattice, bad)
        total_skips += skips
    for _ in range(5):
        bad, skips = violations(*_collinear(g, 20000, sigma), sigma, g)
        assert bad == 0, bad
        total_skips += skips
    assert total_skips > 100000  # the rule does skip entries


def test_codes_rounded_up_are_caught():
    """Planted mistake: codes rounded up from the plain distance difference let the rule skip the nearer
    entry on tight collinear configurations."""
    g = np.random.default_rng(11)
    sigma = f32(0.002)
    bad = sum(violations(*_collinear(g, 20000, sigma), sigma, g, round_up=True)[0] for _ in range(3))
    assert bad > 0


def _lists(g, tgt, pb, r, sigma):
    """Lists built at pb as the kernel builds them: lim from the nearest within r (r2 when none), the <= 8
    nearest by (d2, index) within lim, rho2 = lim when fewer are held, else the 8th d2."""
    r2 = (f32(r) * f32(r)).astype(f32)
    d2 = dist2_rn(pb[:, None, :], tgt[None, :, :])
    idx = np.arange(len(tgt))[None, :].repeat(len(pb), 0)
    order = np.lexsort((idx, d2), axis=1)
    d2s = np.take_along_axis(d2, order, axis=1)
    D = np.where(d2s[:, 0] <= r2, d2s[:, 0], r2).astype(f32)
    s = (fast_sqrt((D * f32(1.0001)).astype(f32), g) + sigma).astype(f32)
    lim = ((s * s).astype(f32) * f32(1.0001)).astype(f32)
    inl = d2s[:, :8] <= lim[:, None]
    m = inl.sum(axis=1)
    rho2 = np.where(m < 8, lim, d2s[:, 7]).astype(f32)
    return order[:, :8], inl, rho2


def test_a_covering_list_holds_the_exact_nearest():
    """The validity test of a list at a new position p: while (sqrt(D') + |p - p_b|)^2 (with the kernel's
    margins) is below rho2, D' being the best listed d2 within r2 (r2 if none), the exact float32 nearest
    neighbour within r, ties to the lower index, is a listed target or there is none.  Random clouds,
    quantised clouds with duplicates (ties at every distance), moves from 0 to 2 sigma."""
    g = np.random.default_rng(5)
    r, sigma = 0.02, f32(0.002)
    r2 = (f32(r) * f32(r)).astype(f32)
    covered_total = 0
    for quant in (None, 0.001):
        tgt = g.uniform(0.0, 0.05, (1500, 3))
        if quant:
            tgt = np.round(tgt / quant) * quant
            tgt[750:900] = tgt[:150]
        tgt = tgt.astype(f32)
        pb = g.uniform(0.005, 0.045, (3000, 3)).astype(f32)
        if quant:
            pb = (np.round(pb / quant) * quant).astype(f32)
        lists, inl, rho2 = _lists(g, tgt, pb, r, sigma)
        for motion in (0.0, 0.3, 1.0, 2.0):
            dirs = g.normal(size=pb.shape)
            dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
            p = (pb + dirs * g.uniform(0.0, motion * float(sigma), (len(pb), 1))).astype(f32)
            if quant and motion == 0.3:
                p = (np.round(p / quant) * quant).astype(f32)
            d2l = dist2_rn(p[:, None, :], tgt[lists])
            d2l = np.where(inl & (d2l <= r2), d2l, np.inf)
            Dp = np.minimum(d2l.min(axis=1), r2).astype(f32)
            moved = dist2_rn(p, pb)
            s = (fast_sqrt((Dp * f32(1.0001)).astype(f32), g) + fast_sqrt((moved * f32(1.0001)).astype(f32), g)).astype(f32)
            covered = (((s * s).astype(f32) * f32(1.0001)).astype(f32) + f32(1e-30)) < rho2
            d2 = dist2_rn(p[:, None, :], tgt[None, :, :])
            d2 = np.where(d2 <= r2, d2, np.inf)
            best = np.lexsort((np.arange(len(tgt))[None, :].repeat(len(p), 0), d2), axis=1)[:, 0]
            has = np.isfinite(d2[np.arange(len(p)), best])
            listed = ((lists == best[:, None]) & inl).any(axis=1)
            assert np.all(~covered | ~has | listed), (quant, motion)
            covered_total += int(covered.sum())
    assert covered_total > 5000  # most lists cover small moves
