"""The index schemes of the temporally blocked kernels (k_step2d, and k_step1d at the end), restated on
the CPU.

A block sweeps a strip of the grid along y with a ring of window rows in shared memory; stage j relaxes
one row per tick, lagging the load by L_1 = |s_1| and stage j - 1 by |s_j| + 1 rows; population k of
logical cell (r, c) after stages 1..j lives at ring row r - acc_j (+y), r + acc_j (-y), r (+-x), column
c - acc_j (+x), c + acc_j (-x); a ring row is reloaded `prefetch` ticks ahead once no stage can read it;
stage j computes only the cells within H - m_j of the output.  This test replays that schedule with every
shared-memory slot tagged by the (plane, row, column, stage) it must hold, on a linear D2Q4 relaxation,
and checks every read against its tag, the absence of same-tick read/write conflicts, and the result
against one pull-shift and relaxation per stage.  The planner's rules (ring = prefetch + max_j (lag_j +
|acc_j|), strips evened over the row, ragged last strip and segment) are the kernel's.
"""
import numpy as np
import pytest

SIGN = [1, 1, -1, -1]  # +x, +y, -x, -y
AXIS = [0, 1, 0, 1]


def relax(fv, omega, a):
    u = fv.sum(0)
    feq = np.stack([u / 4 + a[0] * u / 2, u / 4 + a[1] * u / 2, u / 4 - a[0] * u / 2, u / 4 - a[1] * u / 2])
    return fv + omega * (feq - fv)


def per_stage(f, shifts, omega, a):
    f = f.copy()
    for s in shifts:
        g = np.empty_like(f)
        for k in range(4):
            g[k] = np.roll(f[k], SIGN[k] * s, axis=1 if AXIS[k] == 0 else 0)
        f = relax(g, omega, a)
    return f


def plan(nx, ny, shifts, tx_cap, ly, prefetch=3):
    H = sum(abs(s) for s in shifts)
    lag = acc = E = 0
    for j, s in enumerate(shifts):
        lag += abs(s) + (1 if j > 0 else 0)
        acc += s
        E = max(E, lag + abs(acc))
    hl = (H + 3) // 4 * 4
    nstrips = -(-nx // tx_cap)
    tx = -(-(-(-nx // nstrips)) // 4) * 4
    return dict(H=H, hl=hl, tx=tx, wx=tx + 2 * hl, ly=ly, ring=E + prefetch, prefetch=prefetch,
                nstrips=-(-nx // tx), nsegs=-(-ny // ly))


def blocked(f, shifts, omega, a, p):
    ny, nx = f.shape[1:]
    out = np.full_like(f, np.nan)
    written = np.zeros(f.shape, dtype=int)
    G, H, ring = len(shifts), p["H"], p["ring"]
    lags, ms, accs = [], [], []
    lag = m = acc = 0
    for j, s in enumerate(shifts):
        lag += abs(s) + (1 if j > 0 else 0)
        m += abs(s)
        acc += s
        lags.append(lag), ms.append(m), accs.append(acc)
    for b in range(p["nstrips"] * p["nsegs"]):
        x0, y0 = (b % p["nstrips"]) * p["tx"], (b // p["nstrips"]) * p["ly"]
        tx, ly = min(p["tx"], nx - x0), min(p["ly"], ny - y0)
        wx, nrows = tx + 2 * p["hl"], ly + 2 * H
        val = np.full((ring, 4, p["wx"]), np.nan)
        tag = np.empty((ring, 4, p["wx"]), dtype=object)

        def load(r):
            gy = (y0 - H + r) % ny
            cols = (x0 - p["hl"] + np.arange(wx)) % nx
            for k in range(4):
                val[r % ring, k, :wx] = f[k, gy, cols]
                for c in range(wx):
                    tag[r % ring, k, c] = (k, r, c, 0)

        for r in range(min(p["prefetch"], nrows)):
            load(r)
        for tau in range(ly + H + lags[-1]):
            writes = {}
            for j in range(G):
                r = tau - lags[j]
                if not (ms[j] <= r < nrows - ms[j]):
                    continue
                s, acc = shifts[j], accs[j]
                rows = [r, r - acc, r, r + acc]
                for c in range(p["hl"] - H + ms[j], p["hl"] + tx + H - ms[j]):
                    cols = [c - acc, c, c + acc, c]
                    fv = np.empty(4)
                    for k in range(4):
                        slot = (rows[k] % ring, k, cols[k])
                        assert 0 <= rows[k] and 0 <= cols[k] < wx
                        assert slot not in writes, "read of a slot written in the same tick"
                        er = r - (SIGN[k] * s if AXIS[k] == 1 else 0)
                        ec = c - (SIGN[k] * s if AXIS[k] == 0 else 0)
                        assert tag[slot] == (k, er, ec, j)
                        fv[k] = val[slot]
                    fn = relax(fv, omega, a)
                    if j == G - 1:
                        assert H <= r < H + ly and p["hl"] <= c < p["hl"] + tx
                        gy, gx = y0 + r - H, x0 + c - p["hl"]
                        out[:, gy, gx] = fn
                        written[:, gy, gx] += 1
                    else:
                        for k in range(4):
                            writes[(rows[k] % ring, k, cols[k])] = (fn[k], (k, r, c, j + 1))
            for slot, (v, t) in writes.items():
                val[slot], tag[slot] = v, t
            if tau + p["prefetch"] < nrows:
                load(tau + p["prefetch"])
    assert np.all(written == 1)
    return out


@pytest.mark.parametrize("shape,shifts,tx_cap,ly", [
    ((40, 23), [2, 2], 16, 8),                 # two stages (the headline's group), ragged segment
    ((36, 20), [2, 2, 2, 2, 2, 2], 24, 12),    # six stages, a strip wider than half the row
    ((44, 17), [2, -1, -4, -1, 2, 2], 20, 9),  # the middle of the composite step: negative shifts
    ((24, 13), [1, 2, 2], 8, 13),              # the step's first stage (shift 1), one segment
    ((28, 15), [0, 2], 12, 7),                 # a projection without transport (schemes II-IV)
])
def test_blocked_schedule_matches_per_stage(shape, shifts, tx_cap, ly):
    nx, ny = shape
    f = np.random.default_rng(7).standard_normal((4, ny, nx))
    p = plan(nx, ny, shifts, tx_cap, ly)
    got = blocked(f, shifts, 1.7, (0.2, -0.15), p)
    assert np.abs(got - per_stage(f, shifts, 1.7, (0.2, -0.15))).max() < 1e-12


def fused1d(f, shifts, omega, a, T):
    """The 1D fused step (k_step1d): a tile of T cells and a window of W = T + 2H cells of every plane in
    shared memory; population k of window cell x lives at circular slot (x - o_k) mod W, a stage adds
    sign_k s to o_k and relaxes the cells [m, W - m) in place (m = |s_1| + ... up to this stage), and the
    tile [H, H + T) is written out."""
    n = f.shape[1]
    H = sum(abs(s) for s in shifts)
    out = np.full_like(f, np.nan)
    sign = [1, -1]
    for x0 in range(0, n, T):
        t = min(T, n - x0)
        W = t + 2 * H
        idx = (x0 - H + np.arange(W)) % n
        val = f[:, idx].copy()
        tag = [[(k, i, 0) for i in range(W)] for k in range(2)]
        off, moved = [0, 0], 0
        for st, s in enumerate(shifts):
            off = [off[k] + sign[k] * s for k in range(2)]
            moved += abs(s)
            new = {}
            for x in range(moved, W - moved):
                fv = np.empty(2)
                for k in range(2):
                    slot = (x - off[k]) % W
                    assert tag[k][slot] == (k, x - sign[k] * s, st)
                    fv[k] = val[k, slot]
                u = fv.sum()
                fe = np.array([u / 2 + a * u / 2, u / 2 - a * u / 2])
                fn = fv + omega * (fe - fv)
                for k in range(2):
                    new[(k, (x - off[k]) % W)] = (fn[k], (k, x, st + 1))
            for (k, slot), (v, tg) in new.items():
                val[k, slot], tag[k][slot] = v, tg
        for x in range(H, H + t):
            for k in range(2):
                slot = (x - off[k]) % W
                assert tag[k][slot] == (k, x, len(shifts))
                out[k, x0 + x - H] = val[k, slot]
    return out


def per_stage_1d(f, shifts, omega, a):
    f = f.copy()
    for s in shifts:
        g = np.stack([np.roll(f[0], s), np.roll(f[1], -s)])
        u = g.sum(0)
        fe = np.stack([u / 2 + a * u / 2, u / 2 - a * u / 2])
        f = g + omega * (fe - g)
    return f


@pytest.mark.parametrize("n,T", [(64, 16), (70, 24), (50, 50)])
def test_fused1d_schedule_matches_per_stage(n, T):
    """All 18 stages of a composite step (shifts 1, 2 x 7, -1, -4, -1, 2 x 7) in one window, ragged last
    tile included."""
    shifts = [1] + [2] * 7 + [-1, -4, -1] + [2] * 7
    f = np.random.default_rng(3).standard_normal((2, n))
    got = fused1d(f, shifts, 1.8, 0.3, T)
    assert np.abs(got - per_stage_1d(f, shifts, 1.8, 0.3)).max() < 1e-12
