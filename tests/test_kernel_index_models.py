"""Python models of the index arithmetic of three GPU kernels, checked on the
CPU against brute force: the (G+1)-ary group search, the merge-path split
narrowed by recorded tile samples (k_partition), and the merge step with one
unguarded shared-memory load (merge_tile).  Each model follows its kernel line
by line in plain Python; the GPU tests compare the kernels' outputs with the
oracle, these pin the reasoning the kernels rely on (every probe in range, the
narrowed stretch holding the split, reads within the padded buffer)."""
import random

import pytest


def group_search(lo, hi, G, before):
    """The smallest m in [lo, hi] with before(m) false (hi counts as false),
    found by G lanes probing G evenly spaced points per round (as in
    group_search of sr_device.cuh).  Checks that the lanes' answers form the
    true/false split a warp ballot relies on."""
    rounds = 0
    while hi > lo:
        step = (hi - lo + G) // (G + 1)
        bs = []
        for j in range(G):
            m = lo + (j + 1) * step - 1
            bs.append(m < hi and before(m))
        cnt = sum(bs)
        assert bs == [True] * cnt + [False] * (G - cnt)
        nhi = hi if cnt == G else lo + (cnt + 1) * step - 1
        lo = lo + cnt * step
        hi = min(hi, nhi)
        rounds += 1
    return lo, rounds


@pytest.mark.parametrize("G", [1, 2, 4, 8, 32])
def test_group_search_finds_the_split(G):
    rng = random.Random(G)
    for _ in range(2000):
        lo = rng.randint(0, 50)
        hi = lo + rng.randint(0, 5000)
        ans = rng.randint(lo, hi)
        got, rounds = group_search(lo, hi, G, lambda m: m < ans)
        assert got == ans
        # every round keeps at most 1/(G+1) of the stretch (plus one)
        bound = 0
        n = hi - lo
        while n > 0:
            n = (n + G) // (G + 1) - 1 if n > G else 0
            bound += 1
        assert rounds <= bound + 1


def _stable_split(A, B, d):
    """Keys of A among the first d outputs of the stable merge (A first on ties)."""
    i = j = 0
    for _ in range(d):
        if j >= len(B) or (i < len(A) and not (B[j] < A[i])):
            i += 1
        else:
            j += 1
    return i


def test_sample_guided_split_equals_merge_path():
    """k_partition: a coarse search over the first key of A's tiles and the
    last key of B's tiles, then a fine search inside the one tile stretch the
    samples leave, gives the merge-path split at every output tile boundary;
    the samples it reads are the keys the direct test would read."""
    rng = random.Random(7)
    for trial in range(1500):
        nv = rng.choice([3, 4, 5, 7, 8])
        ts = nv * rng.choice([1, 2, 4])
        n = rng.randint(1, 60 * nv)
        w = ts << rng.randint(0, 4)
        vals = rng.choice([3, 10, 1000])
        data = [rng.randrange(vals) for _ in range(n)]
        for s0 in range(0, n, w):
            data[s0:s0 + w] = sorted(data[s0:s0 + w])
        mtiles = (n + nv - 1) // nv
        samp = []
        for t in range(mtiles):
            seg = data[t * nv:min(n, (t + 1) * nv)]
            samp += [seg[0], seg[-1]]
        G = rng.choice([1, 2, 4, 32])
        for b in range(mtiles + 1):
            out = min(b * nv, n)
            pb = (out // (2 * w)) * (2 * w)
            a_beg, a_end = pb, min(pb + w, n)
            b_beg, b_end = a_end, min(pb + 2 * w, n)
            na, nb, d = a_end - a_beg, b_end - b_beg, out - pb
            lo, hi = max(0, d - nb), min(d, na)
            A, B = data[a_beg:a_end], data[b_beg:b_end]
            if out < n and hi > lo:
                assert d % nv == 0 and a_beg % nv == 0 and b_beg % nv == 0
                jlo, jhi, dj = (lo + nv - 1) // nv, (hi - 1) // nv, d // nv
                ta, tb = a_beg // nv, b_beg // nv

                def coarse(j):
                    x, y = samp[2 * (ta + j)], samp[2 * (tb + dj - j - 1) + 1]
                    assert x == A[j * nv] and y == B[d - 1 - j * nv]
                    return not (y < x)
                jt, _ = group_search(jlo, jhi + 1, G, coarse)
                if jt > jlo:
                    lo = max(lo, (jt - 1) * nv + 1)
                if jt <= jhi:
                    hi = min(hi, jt * nv)
                assert hi - lo <= nv
            sp, _ = group_search(lo, hi, G, lambda m: not (B[d - 1 - m] < A[m]))
            assert sp == _stable_split(A, B, d), trial


def _serial_merge(s, a, a_end, b, b_end, ipt, slack):
    """merge_tile's per-thread merge step; slack: one unguarded load per step.
    Returns the outputs and the largest index read."""
    out, mx = [], -1
    if slack:
        ak, bk = s[a], s[b]
        mx = max(a, b)
    else:
        ak = s[a] if a < a_end else 0
        bk = s[b] if b < b_end else 0
    for _ in range(ipt):
        take_a = b >= b_end or (a < a_end and not (bk < ak))
        out.append(ak if take_a else bk)
        if slack:
            nx = (a if take_a else b) + 1
            mx = max(mx, nx)
            if take_a:
                a, ak = nx, s[nx]
            else:
                b, bk = nx, s[nx]
        elif take_a:
            a += 1
            if a < a_end:
                ak = s[a]
        else:
            b += 1
            if b < b_end:
                bk = s[b]
    return out, mx


def test_one_load_merge_step_matches_and_stays_in_the_padding():
    """The unguarded step gives the same outputs wherever they are written and
    never reads past max(a_end, b_end) + IPT -- the IPT + 8 keys of padding
    the merge kernels allocate after the staged keys."""
    rng = random.Random(3)
    for _ in range(20000):
        ipt = rng.randint(1, 9)
        na, nb = rng.randint(0, 20), rng.randint(0, 20)
        A = sorted(rng.randrange(5) for _ in range(na))
        B = sorted(rng.randrange(5) for _ in range(nb))
        sa, pad = rng.randint(0, 3), rng.randint(0, 3)
        s = [99] * sa + A + [98] * pad + B + [77] * (ipt + 8)
        sb = sa + na + pad
        diag = rng.randint(0, na + nb)
        lo, hi = max(0, diag - nb), min(diag, na)
        while lo < hi:
            m = (lo + hi) // 2
            if not (B[diag - 1 - m] < A[m]):
                lo = m + 1
            else:
                hi = m
        o1, _ = _serial_merge(s, sa + lo, sa + na, sb + diag - lo, sb + nb, ipt, False)
        o2, mx = _serial_merge(s, sa + lo, sa + na, sb + diag - lo, sb + nb, ipt, True)
        valid = min(ipt, na + nb - diag)
        assert o1[:valid] == o2[:valid]
        assert mx <= max(sa + na, sb + nb) + ipt


# ------------------------------------------------------------ 4-way steps

class _Checked:
    """A list whose reads must fall in [lo, hi) (asserts, naming the buffer)."""

    def __init__(self, data, name, lo=0, hi=None):
        self.d, self.name, self.lo = data, name, lo
        self.hi = len(data) if hi is None else hi

    def __getitem__(self, i):
        assert self.lo <= i < self.hi, (self.name, i, self.lo, self.hi)
        return self.d[i]


def _pair_tile(split1, P, nv, j):
    x_beg, x_end, y_end, t0, ln = P
    assert 0 <= j * nv < ln
    xs = split1[t0 + j]
    o1 = min((j + 1) * nv, ln)
    xe = x_end if o1 == ln else split1[t0 + j + 1]
    ys = x_end + j * nv - (xs - x_beg)
    ye = x_end + o1 - (xe - x_beg)
    assert x_beg <= xs <= xe <= x_end and x_end <= ys <= ye <= y_end
    return xs, xe, ys, ye


def _pair_key(src, split1, P, nv, m):
    j = m // nv
    xs, xe, ys, ye = _pair_tile(split1, P, nv, j)
    r = m - j * nv
    nx, ny = xe - xs, ye - ys
    X, Y = _Checked(src, "X", xs, xe), _Checked(src, "Y", ys, ye)
    lo, hi = max(0, r + 1 - ny), min(r + 1, nx)
    while lo < hi:
        mid = (lo + hi) >> 1
        if not (Y[ys + r - mid] < X[xs + mid]):
            lo = mid + 1
        else:
            hi = mid
    v = None
    if lo > 0:
        v = X[xs + lo - 1]
    if r - lo >= 0:
        y = Y[ys + r - lo]
        v = y if v is None or v < y else v
    return v


def _pair_split(src, split1, P, nv, x):
    x_beg, x_end, y_end, t0, ln = P
    if x >= ln:
        return x_end - x_beg
    j = x // nv
    xs, xe, ys, ye = _pair_tile(split1, P, nv, j)
    r = x - j * nv
    nx, ny = xe - xs, ye - ys
    X, Y = _Checked(src, "X", xs, xe), _Checked(src, "Y", ys, ye)
    lo, hi = max(0, r - ny), min(r, nx)
    while lo < hi:
        mid = (lo + hi) >> 1
        if not (Y[ys + r - 1 - mid] < X[xs + mid]):
            lo = mid + 1
        else:
            hi = mid
    return xs + lo - x_beg


def _pair_first(src, split1, P, nv, j):
    xs, xe, ys, ye = _pair_tile(split1, P, nv, j)
    if xs < xe and (ys >= ye or not (src[ys] < src[xs])):
        return src[xs]
    return src[ys]


def _pair_last(src, split1, P, nv, j):
    xs, xe, ys, ye = _pair_tile(split1, P, nv, j)
    v = src[xe - 1] if xe > xs else None
    if ye > ys:
        v = src[ye - 1] if v is None or v < src[ye - 1] else v
    return v


def _partition4(src, n, w, nv, split1, b, G):
    """k_partition4 for boundary b: where tile b's share of A, B, C, D starts."""
    if b * nv >= n:
        return [n] * 4
    out = b * nv
    G0 = (out // (4 * w)) * (4 * w)
    e = [min(G0 + i * w, n) for i in range(5)]
    AB = (e[0], e[1], e[2], e[0] // nv, e[2] - e[0])
    CD = (e[2], e[3], e[4], e[2] // nv, e[4] - e[2])
    d = out - G0
    assert d % nv == 0
    lo, hi = max(0, d - CD[4]), min(d, AB[4])
    if hi > lo:
        jlo, jhi, dj = (lo + nv - 1) // nv, (hi - 1) // nv, d // nv
        if jlo <= jhi:
            jt, _ = group_search(jlo, jhi + 1, G, lambda j: not (
                _pair_last(src, split1, CD, nv, dj - j - 1) < _pair_first(src, split1, AB, nv, j)))
            # the coarse probe equals the fine one at m = j * nv
            for j in range(jlo, jhi + 1):
                m = j * nv
                assert _pair_last(src, split1, CD, nv, dj - j - 1).v == _pair_key(src, split1, CD, nv, d - 1 - m).v
                assert _pair_first(src, split1, AB, nv, j).v == _pair_key(src, split1, AB, nv, m).v
            if jt > jlo:
                lo = max(lo, (jt - 1) * nv + 1)
            if jt <= jhi:
                hi = min(hi, jt * nv)
        lo, _ = group_search(lo, hi, G, lambda m: not (
            _pair_key(src, split1, CD, nv, d - 1 - m) < _pair_key(src, split1, AB, nv, m)))
    x = lo
    a = _pair_split(src, split1, AB, nv, x)
    c = _pair_split(src, split1, CD, nv, d - x)
    return [e[0] + a, e[1] + (x - a), e[2] + c, e[3] + (d - x - c)]


def _serial(s, a, a_end, b, b_end, ipt, sw=None, c=None):
    """serial_merge_slack (sw None) or serial_merge_switch: IPT outputs from
    shared memory s (reads checked against its size)."""
    out, ix = [], []
    if sw is None:
        ak, bk = s[a], s[b]
        for _ in range(ipt):
            take_a = b >= b_end or (a < a_end and not (bk < ak))
            out.append(ak if take_a else bk)
            ix.append(a if take_a else b)
            nx = (a if take_a else b) + 1
            nk = s[nx]
            if take_a:
                a, ak = nx, nk
            else:
                b, bk = nx, nk
        return out, ix
    for i in range(ipt):
        if i == sw:
            a, a_end, b, b_end = c
        take_a = b >= b_end or (a < a_end and not (s[b] < s[a]))
        at = a if take_a else b
        out.append(s[at])
        ix.append(at)
        if take_a:
            a += 1
        else:
            b += 1
    return out, ix


def _merge_path(s, a0, na, b0, nb, diag):
    lo, hi = max(0, diag - nb), min(diag, na)
    while lo < hi:
        mid = (lo + hi) >> 1
        if not (s[b0 + diag - 1 - mid] < s[a0 + mid]):
            lo = mid + 1
        else:
            hi = mid
    return lo


def _merge_tile4(src, n, out0, cnt, beg, ln, NT, IPT, bulk):
    """merge_tile4 with 4-key group staging (STAGE_VEC / STAGE_BULK) and its
    two merge levels; keys are (value, run, position) so ties show order."""
    NV = NT * IPT
    SV = NV + 32
    size = SV + IPT + 8                           # keys readable in shared memory
    g0 = [b & ~3 for b in beg]
    first = [0]
    for i in range(4):
        ng = (((beg[i] + ln[i] + 3) & ~3) - g0[i]) >> 2 if ln[i] > 0 else 0
        first.append(first[-1] + ng)
    assert 4 * first[4] <= SV
    pos = [4 * first[i] + (beg[i] - g0[i]) for i in range(4)]
    smem = [_K(float("inf"), 9, 9)] * size        # garbage beyond the staged keys
    n4 = n & ~3
    for i in range(4):
        ge = g0[i] + 4 * (first[i + 1] - first[i])
        if bulk:
            hi = min(ge, n4)
            if hi > g0[i]:
                assert g0[i] % 4 == 0 and hi % 4 == 0 and 0 <= g0[i] and hi <= n   # 16-byte spans
                for g in range(g0[i], hi):
                    smem[4 * first[i] + g - g0[i]] = src[g]
            if ln[i] > 0 and beg[i] + ln[i] > n4:
                for g in range(max(n4, g0[i]), beg[i] + ln[i]):
                    assert g - max(n4, g0[i]) < NT                    # one key per thread
                    smem[4 * first[i] + g - g0[i]] = src[g]
        else:
            for g in range(g0[i], ge):
                if g < n:
                    smem[4 * first[i] + g - g0[i]] = src[g]
    s = _Checked(smem, "smem")
    lab = ln[0] + ln[1]
    regs = []
    for t in range(NT):
        o = min(t * IPT, cnt)
        if o + IPT <= lab:
            sp = _merge_path(s, pos[0], ln[0], pos[1], ln[1], o)
            k, _ = _serial(s, pos[0] + sp, pos[0] + ln[0], pos[1] + o - sp, pos[1] + ln[1], IPT)
        elif o >= lab:
            oc = o - lab
            sp = _merge_path(s, pos[2], ln[2], pos[3], ln[3], oc)
            k, _ = _serial(s, pos[2] + sp, pos[2] + ln[2], pos[3] + oc - sp, pos[3] + ln[3], IPT)
        else:
            sp = _merge_path(s, pos[0], ln[0], pos[1], ln[1], o)
            k, _ = _serial(s, pos[0] + sp, pos[0] + ln[0], pos[1] + o - sp, pos[1] + ln[1], IPT, sw=lab - o,
                           c=(pos[2], pos[2] + ln[2], pos[3], pos[3] + ln[3]))
        regs.extend(k)
    smem2 = regs + [_K(float("inf"), 9, 9)] * (size - len(regs))
    s2 = _Checked(smem2, "smem")
    for part in (smem2[:lab], smem2[lab:cnt]):
        assert [k.full() for k in part] == sorted(k.full() for k in part)
    res = []
    for t in range(NT):
        diag = min(t * IPT, cnt)
        sp = _merge_path(s2, 0, lab, lab, cnt - lab, diag)
        k, _ = _serial(s2, sp, lab, lab + diag - sp, cnt, IPT)
        res.extend(k)
    return res[:cnt]


class _K:
    """A key that compares by value alone (as the kernels do) and remembers
    its run and original position, so the output's tie order can be checked."""
    __slots__ = ("v", "run", "pos")

    def __init__(self, v, run, pos):
        self.v, self.run, self.pos = v, run, pos

    def __lt__(self, o):
        return self.v < o.v

    def full(self):
        return (self.v, self.run, self.pos)


@pytest.mark.parametrize("seed", range(6))
def test_four_way_step_model(seed):
    """Block-sorted tiles merged by the step schedule of sr_plain.cuh (a 2-way
    step first when the level count is odd, then 4-way steps) with the split
    tables and merge tiles of the 4-way kernels modelled: every read inside
    its run window or the shared buffer, every output tile equal to the stable
    merge of its group (ties: A, B, C, D, then position)."""
    rng = random.Random(100 + seed)
    NT, IPT = 8, 3
    nv = NT * IPT
    ts = 2 * nv
    for trial in range(12):
        n = rng.choice([rng.randint(1, 10 * ts), rng.randint(10 * ts, 70 * ts)])
        alpha = rng.choice([3, 50, 10 ** 6])
        vals = [rng.randrange(alpha) for _ in range(n)]
        # keys compare by value; each remembers its original position
        tiles = (n + ts - 1) // ts
        keys = []
        for t in range(tiles):
            idx = sorted(range(t * ts, min(n, (t + 1) * ts)), key=lambda i: (vals[i], i))
            keys.extend(_K(vals[i], 0, i) for i in idx)
        levels = 0
        while (1 << levels) < tiles:
            levels += 1
        steps = (levels + 1) // 2
        for st in range(steps):
            if levels & 1 and st == 0:
                l0, nl = 0, 1
            else:
                l0, nl = (levels & 1) + 2 * (st - (levels & 1)), 2
            w = ts << l0
            if nl == 1:
                new = []
                for p0 in range(0, n, 2 * w):
                    new.extend(sorted(keys[p0:min(n, p0 + 2 * w)], key=lambda k: (k.v, k.pos)))
                keys = new
                continue
            mt = (n + nv - 1) // nv
            # split1: the 2-way split (k_partition) of every tile boundary
            split1 = []
            for b in range(mt + 1):
                out = min(b * nv, n)
                pb = (out // (2 * w)) * (2 * w)
                A, B = keys[pb:min(pb + w, n)], keys[min(pb + w, n):min(pb + 2 * w, n)]
                split1.append(pb + _stable_split(A, B, out - pb))
            G = rng.choice([1, 2, 4, 8])
            split4 = [_partition4(keys, n, w, nv, split1, b, G) for b in range(mt + 1)]
            # tag every key with its run in the group (A..D) for the tie order
            tagged = [_K(k.v, (g % (4 * w)) // w, k.pos) for g, k in enumerate(keys)]
            new = []
            for b in range(mt):
                out0, out1 = b * nv, min(b * nv + nv, n)
                G0 = (out0 // (4 * w)) * (4 * w)
                last = out1 == min(G0 + 4 * w, n)
                beg = split4[b]
                end = [min(G0 + (i + 1) * w, n) for i in range(4)] if last else split4[b + 1]
                ln = [end[i] - beg[i] for i in range(4)]
                assert sum(ln) == out1 - out0 and min(ln) >= 0
                got = _merge_tile4(tagged, n, out0, out1 - out0, beg, ln, NT, IPT, bulk=(b + trial) % 2 == 0)
                grp = sorted(k.full() for k in tagged[G0:min(G0 + 4 * w, n)])
                assert [k.full() for k in got] == grp[out0 - G0:out1 - G0], (n, w, b)
                new.extend(got)
            keys = new
            # within a run, positions ascend on ties (every earlier step was stable)
        assert [(k.v, k.pos) for k in keys] == sorted((v, i) for i, v in enumerate(vals))
