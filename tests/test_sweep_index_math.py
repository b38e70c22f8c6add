"""The sweep's run bookkeeping against brute force (CPU, no GPU).

A run of an edge point is the set of global steps s in [s_lo, s_hi] whose
spindle phase index (s mod S) lies in the arc m0 .. m0+len-1 (mod S): the
steps at which that point can be over a tile (Section 2.3's time loop,
restricted per tile). The kernels never list these steps; they derive them
from the run's iteration record (first occurrence, offset into it, lengths of
the first and last occurrences, last revolution) by integer arithmetic with
float-reciprocal divisions. This test models that arithmetic -- the record,
the item form's incremental (revolution, phase offset) walk of 8-lane groups
taking items hl and hl + 8 of every 16, and the phase form's range of
revolutions per phase offset -- and checks both against the brute-force set
of steps, item by item, over random runs."""
import numpy as np

f32 = np.float32
L = 8  # lanes per run in the item form


def imod_pos(a, S):
    q = int(np.floor(f32(a) * (f32(1.0) / f32(S))))
    r = a - q * S
    while r < 0:
        r += S
    while r >= S:
        r -= S
    return r


def idiv_floor(a, S):
    q = int(f32(a) * (f32(1.0) / f32(S)))
    while q * S > a:
        q -= 1
    while (q + 1) * S <= a:
        q += 1
    return q


def run_iter(m0, ln, s_lo, s_hi, S):
    base = s_lo - imod_pos(s_lo - m0, S)
    if base + ln - 1 < s_lo:
        base += S
    if base > s_hi:
        return None
    f0, e0 = max(base, s_lo), min(base + ln - 1, s_hi)
    first_off, len0 = f0 - base, e0 - f0 + 1
    k_last = idiv_floor(s_hi - base, S)
    if k_last == 0:
        len_last, total = 0, len0
    else:
        ol = base + k_last * S
        len_last = min(ol + ln - 1, s_hi) - ol + 1
        total = len0 + (k_last - 1) * ln + len_last
    return dict(occ0=base, first_off=first_off, len0=len0, k_last=k_last, len_last=len_last, total=total)


def divmod_small(v, ln, inv_len):
    d = int(f32(v) * inv_len)  # truncation toward zero, v >= 0
    d += 1 if (d + 1) * ln <= v else 0
    d -= 1 if d * ln > v else 0
    return d, v - d * ln


def item_walk(r, m0, ln, S, U=2):
    """Steps and phases the item form visits, by item index: lane hl's U
    chains start at items hl, hl + L, ... (revolution q and phase offset o
    from one division each), then carry their phase index mn (m0 + o, below
    2S: the table holds two turns) and their steps after the run's first item
    dn, both advanced by U L items per iteration, the phase wrapping within
    the run's arc (and adding the arc's gap to the steps)."""
    inv_len = f32(1.0) / f32(ln)
    gap = S - ln
    s_a = r["occ0"] + r["first_off"]
    dul, rul = divmod_small(U * L, ln, inv_len)
    dl, rl = divmod_small(L, ln, inv_len)
    out = {}
    tot = r["total"]
    m_end, dn_step = m0 + ln, U * L + dul * gap
    for hl in range(L):
        q, o = divmod_small(hl + r["first_off"], ln, inv_len)
        mn, dn = [], []
        for k in range(U):
            if k > 0:
                o += rl
                q += dl
                if o >= ln:
                    o -= ln
                    q += 1
            mn.append(m0 + o)
            dn.append(hl + k * L + q * gap)
        base = 0
        while base < tot:
            for k in range(U):
                t = base + hl + k * L
                assert mn[k] < 2 * S
                if t < tot:
                    m = mn[k] - S if mn[k] >= S else mn[k]
                    out[t] = (s_a + dn[k], m)
                mn[k] += rul
                dn[k] += dn_step
                if mn[k] >= m_end:
                    mn[k] -= ln
                    dn[k] += gap
            base += U * L
    return out


def phase_walk(r, ln, S):
    """Steps the phase form visits: per phase offset, revolutions kb..ke."""
    f0, f1 = r["first_off"], r["first_off"] + r["len0"]
    steps = []
    for off in range(ln):
        kb = 0 if f0 <= off < f1 else 1
        ke = 0 if r["k_last"] == 0 else (r["k_last"] if off < r["len_last"] else r["k_last"] - 1)
        steps.extend(r["occ0"] + k * S + off for k in range(kb, ke + 1))
    return sorted(steps)


def test_run_items_and_phases_match_brute_force():
    rng = np.random.default_rng(2603)
    checked = 0
    for _ in range(3000):
        S = int(rng.integers(1, 4000))
        m0 = int(rng.integers(0, S))
        ln = int(rng.integers(1, S + 1))
        s_lo = int(rng.integers(0, 10**6))
        s_hi = s_lo + int(rng.integers(0, 6000 if rng.random() < 0.8 else 40))
        brute = [s for s in range(s_lo, s_hi + 1) if (s - m0) % S < ln]
        r = run_iter(m0, ln, s_lo, s_hi, S)
        if r is None or r["total"] <= 0:
            assert not brute
            continue
        assert r["total"] == len(brute)
        for U in (2, 3):
            items = item_walk(r, m0, ln, S, U)
            assert sorted(items) == list(range(r["total"]))
            assert [items[t][0] for t in range(r["total"])] == brute  # item t is the t-th step of the run
            assert all(m == s % S for s, m in items.values())         # and its phase index
        assert phase_walk(r, ln, S) == brute
        checked += len(brute)
    assert checked > 10**6


def fma32(a, b, c):
    """fmaf of float32 arrays: the product is exact in float64, one rounding."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def test_phase_form_revolution_range_contains_every_revolution_over_the_tile():
    """Phase form: for one phase offset, revolution k of a run is
    ds_k = d0 + k S steps after the run's first item, at tile-local x (cells)
    fma(ds_k, fs, dxA) + px in FP32. The kernel visits k in
    [max(kb, ceil(fma(-x0, r, lo r))), min(ke, floor(fma(-x0, r, hi r)))],
    r = 1 / (S fs), x0 = fma(d0, fs, dxA) + px, with (lo, hi) = (-(M + 1),
    txc + M) (swapped on a return pass, fs < 0), in FP32. Coordinates are centred on cells
    (the cell is the nearest integer), so every revolution whose FP32 x
    rounds into the tile widened by M cells -- x in [-M - 1/2, txc - 1 + M
    + 1/2] -- must be visited, for both feed directions."""
    rng = np.random.default_rng(61)
    hit = 0
    for _ in range(4000):
        S = int(rng.integers(1, 40000))
        fs = f32(10.0 ** rng.uniform(-4.0, 1.0) * (1 if rng.random() < 0.5 else -1))  # cells per step
        txc = int(rng.integers(1, 1025))
        M = int(rng.integers(1, 4))
        kb, ke = int(rng.integers(0, 2)), int(rng.integers(0, 400))
        if ke < kb or abs(float(fs)) * S * ke > 1e6:
            continue
        d0 = f32(-int(rng.integers(0, S)) + int(rng.integers(0, S)))
        px = f32(rng.uniform(-3000.0, 3000.0))
        # an anchor that brings some revolutions over the tile
        k_mid = rng.uniform(kb, ke + 1)
        dxa = f32(rng.uniform(-M - 2, txc + M + 2) - float(px) - (float(d0) + k_mid * S) * float(fs))
        back = fs < 0
        lo, hi = f32(-(M + 1.0)), f32(txc + M)
        k_lo, k_hi = (hi, lo) if back else (lo, hi)
        inv_rev = f32(1.0) / (f32(S) * fs)
        x0 = (fma32(np.array([d0]), np.array([fs]), np.array([dxa]))[0] + px).astype(f32)
        klo_c, khi_c = f32(k_lo * inv_rev), f32(k_hi * inv_rev)
        k0 = max(kb, int(np.ceil(fma32(np.array([-x0]), np.array([inv_rev]), np.array([klo_c]))[0])))
        k1 = min(ke, int(np.floor(fma32(np.array([-x0]), np.array([inv_rev]), np.array([khi_c]))[0])))
        ks = np.arange(kb, ke + 1)
        ds = (f32(d0) + ks.astype(np.float64) * S).astype(f32)
        xs = (fma32(ds, np.full(ks.size, fs, f32), np.full(ks.size, dxa, f32)) + px).astype(f32).astype(np.float64)
        over = ks[(xs >= -M - 0.5) & (xs <= txc - 1 + M + 0.5)]
        hit += over.size
        ok = over.size == 0 or (over.min() >= k0 and over.max() <= k1)
        assert ok, (S, fs, float(x0), over, k0, k1)
        # and the range is tight: its revolutions span no more x than the
        # widened tile (txc + 2M + 1 cells), up to float rounding
        if k1 > k0:
            assert (k1 - k0) * abs(float(fs)) * S <= (txc + 2 * M + 1) * (1 + 1e-5) + 1e-3
    assert hit > 1000


def rev_range(v0, rev, lo, hi, kb, ke):
    """The tilted phase form's revolution range of one coordinate (FP32)."""
    if abs(float(rev)) < 1e-4:
        drift = f32(abs(float(rev)) * (ke - kb + 1) + 1.0)
        ok = (v0 >= lo - drift) and (v0 <= hi + drift)
        return (kb, ke) if ok else (1, 0)
    inv = f32(1.0) / rev
    a, b = f32((lo - v0) * inv), f32((hi - v0) * inv)
    return max(kb, int(np.ceil(min(a, b)))), min(ke, int(np.floor(max(a, b))))


def test_tilted_phase_form_revolution_range_covers_the_tile():
    """Tilted phase form: revolution k of a phase offset sits at (FP32)
    x = fma(ds_k, fsx, dxA) + px, y = fma(ds_k, fsy, dyA) + py with
    ds_k = d0 + k S; the kernel visits the intersection of the ranges of x in
    [-(M + 1), txc + M] and y in [-(M + 1), tyc + M] with the run's [kb, ke].
    Every revolution whose x and y round into the tile widened by M cells
    must be visited, at any feed direction (including ones where a
    coordinate barely moves per revolution) and both pass directions."""
    rng = np.random.default_rng(67)
    hit = 0
    for _ in range(6000):
        S = int(rng.integers(1, 40000))
        fs = 10.0 ** rng.uniform(-4.0, 1.0)
        phi = rng.choice([rng.uniform(0, 2 * np.pi), 0.0, np.pi / 2, rng.uniform(-1e-7, 1e-7),
                          np.pi / 2 + rng.uniform(-1e-7, 1e-7)])
        sign = 1 if rng.random() < 0.5 else -1
        fsx, fsy = f32(sign * fs * np.cos(phi)), f32(sign * fs * np.sin(phi))
        txc, tyc = int(rng.integers(1, 1025)), int(rng.integers(1, 200))
        M = int(rng.integers(1, 4))
        kb, ke = int(rng.integers(0, 2)), int(rng.integers(0, 300))
        if ke < kb or fs * S * ke > 1e6:
            continue
        d0 = f32(-int(rng.integers(0, S)) + int(rng.integers(0, S)))
        px, py = f32(rng.uniform(-3000.0, 3000.0)), f32(rng.uniform(-3000.0, 3000.0))
        k_mid = rng.uniform(kb, ke + 1)
        dxa = f32(rng.uniform(-M - 2, txc + M + 2) - float(px) - (float(d0) + k_mid * S) * float(fsx))
        dya = f32(rng.uniform(-M - 2, tyc + M + 2) - float(py) - (float(d0) + k_mid * S) * float(fsy))
        rev_x, rev_y = f32(f32(S) * fsx), f32(f32(S) * fsy)
        x0 = (fma32(np.array([d0]), np.array([fsx]), np.array([dxa]))[0] + px).astype(f32)
        y0 = (fma32(np.array([d0]), np.array([fsy]), np.array([dya]))[0] + py).astype(f32)
        kx0, kx1 = rev_range(x0, rev_x, f32(-(M + 1.0)), f32(txc + M), kb, ke)
        ky0, ky1 = rev_range(y0, rev_y, f32(-(M + 1.0)), f32(tyc + M), kb, ke)
        k0, k1 = max(kx0, ky0), min(kx1, ky1)
        ks = np.arange(kb, ke + 1)
        ds = (f32(d0) + ks.astype(np.float64) * S).astype(f32)
        xs = (fma32(ds, np.full(ks.size, fsx, f32), np.full(ks.size, dxa, f32)) + px).astype(f32)
        ys = (fma32(ds, np.full(ks.size, fsy, f32), np.full(ks.size, dya, f32)) + py).astype(f32)
        ix, iy = np.rint(xs.astype(np.float64)), np.rint(ys.astype(np.float64))
        over = ks[(ix >= -M) & (ix <= txc - 1 + M) & (iy >= -M) & (iy <= tyc - 1 + M)]
        hit += over.size
        assert over.size == 0 or (over.min() >= k0 and over.max() <= k1), (S, float(fsx), float(fsy), over, k0, k1)
    assert hit > 1000


def test_plan_threads_take_each_point_and_phase_once():
    """Planning: thread t of a grid of `stride` threads takes the edge points
    t, t + stride, ... below NE, and the phase-table entries from
    t - (NE mod stride) (plus stride where that is negative) in steps of
    stride below S. Every point and every phase entry is built exactly once,
    and a grid of at least NE + S threads gives each thread one item."""
    rng = np.random.default_rng(5)
    cases = [(800, 3600, 4416), (800, 3600, 64), (2, 5, 7), (1000, 300, 640), (3, 3, 64), (1, 1, 1)]
    cases += [(int(rng.integers(1, 3000)), int(rng.integers(1, 8000)), int(rng.integers(1, 9000))) for _ in range(300)]
    for NE, S, stride in cases:
        points = np.zeros(NE, np.int64)
        phases = np.zeros(S, np.int64)
        per_thread = np.zeros(stride, np.int64)
        for first in range(stride):
            idx = np.arange(first, NE, stride)
            points[idx] += 1
            m0 = first - NE % stride
            if m0 < 0:
                m0 += stride
            ms = np.arange(m0, S, stride)
            phases[ms] += 1
            per_thread[first] = idx.size + ms.size
        assert (points == 1).all() and (phases == 1).all(), (NE, S, stride)
        if stride >= NE + S:
            assert per_thread.max() <= 1, (NE, S, stride)
