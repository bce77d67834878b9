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
    xs = split1[t0 + j][0]
    o1 = min((j + 1) * nv, ln)
    xe = x_end if o1 == ln else split1[t0 + j + 1][0]
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


def _nrun_pos(rs0, nruns, q, ts, n):
    return n if q >= nruns else min(rs0[q] * ts, n)


def _nrun_of(rs0, nruns, tiles, t):
    if nruns == tiles:
        return t
    lo, hi = 0, nruns - 1
    while lo < hi:
        mid = (lo + hi + 1) >> 1
        if rs0[mid] <= t:
            lo = mid
        else:
            hi = mid - 1
    assert rs0[lo] <= t < rs0[lo + 1]
    return lo


def _runs(lo_, hi_, tiles, fan):
    """k_runs: natural runs of whole tiles and the steps they need."""
    rs0 = [t for t in range(tiles) if t == 0 or hi_[t - 1] > lo_[t]]
    nruns = len(rs0)
    rs0.append(tiles)
    steps, m = 0, nruns
    while m > 1:
        m = (m + fan - 1) // fan
        steps += 1
    return rs0, nruns, steps


def _partition2(src, n, ts, tiles, nv, rs0, nruns, span, b):
    """k_partition for boundary b: (split, a_beg, a_end, b_end)."""
    out = b * nv
    if out >= n:
        return (n, n, n, n)
    q = _nrun_of(rs0, nruns, tiles, out // ts)
    p0 = (q // (2 * span)) * (2 * span)
    a_beg = _nrun_pos(rs0, nruns, p0, ts, n)
    a_end = _nrun_pos(rs0, nruns, p0 + span, ts, n)
    b_end = _nrun_pos(rs0, nruns, p0 + 2 * span, ts, n)
    assert a_beg <= out < b_end and a_beg % nv == 0 and a_end % ts == 0 or a_end == n
    A = _Checked(src, "A", a_beg, a_end)
    B = _Checked(src, "B", a_end, b_end)
    d = out - a_beg
    lo, hi = max(0, d - (b_end - a_end)), min(d, a_end - a_beg)
    while lo < hi:                                 # the fine search (samples only narrow it)
        mid = (lo + hi) >> 1
        if not (B[a_end + d - 1 - mid] < A[a_beg + mid]):
            lo = mid + 1
        else:
            hi = mid
    return (a_beg + lo, a_beg, a_end, b_end)


def _partition4(src, n, ts, tiles, nv, rs0, nruns, span, split1, b, G):
    """k_partition4 for boundary b: the four window starts and run ends."""
    out = b * nv
    if out >= n:
        return [n] * 8
    q = _nrun_of(rs0, nruns, tiles, out // ts)
    g0 = (q // (4 * span)) * (4 * span)
    e = [_nrun_pos(rs0, nruns, g0 + i * span, ts, n) for i in range(5)]
    AB = (e[0], e[1], e[2], e[0] // nv, e[2] - e[0])
    CD = (e[2], e[3], e[4], e[2] // nv, e[4] - e[2])
    d = out - e[0]
    assert d % nv == 0 and 0 <= d < e[4] - e[0]
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
    x, a, c = _ab_cd_split(src, split1, AB, CD, nv, d, lo, hi, G)
    # the same split by plain searches: every probe's keys searched in full
    want, _ = group_search(lo, hi, G, lambda m: not (
        _pair_key(src, split1, CD, nv, d - 1 - m) < _pair_key(src, split1, AB, nv, m)))
    assert x == want
    assert a == _pair_split(src, split1, AB, nv, x) and c == _pair_split(src, split1, CD, nv, d - x)
    return [e[0] + a, e[1] + (x - a), e[2] + c, e[3] + (d - x - c)] + e[1:]


def _pair_count_at_tile(split1, P, nv, j):
    x_beg, x_end, y_end, t0, ln = P
    if j <= 0:
        return 0
    if j * nv >= ln:
        return x_end - x_beg
    return split1[t0 + j][0] - x_beg


def _pair_count(src, P, q, x):
    """pair_count: S_P(x) searched inside the anchors q = [xl, sl, xh, sh]."""
    x_beg, x_end, y_end, t0, ln = P
    xl, sl, xh, sh = q
    assert xl <= x <= xh
    nx, ny = x_end - x_beg, y_end - x_end
    X, Y = _Checked(src, "X", x_beg, x_end), _Checked(src, "Y", x_end, y_end)
    lo = max(sl, sh - (xh - x), 0, x - ny)
    hi = min(sh, sl + (x - xl), x, nx)
    assert lo <= hi
    while lo < hi:
        mid = (lo + hi) >> 1
        if not (Y[x_end + x - 1 - mid] < X[x_beg + mid]):
            lo = mid + 1
        else:
            hi = mid
    return lo


def _ab_cd_split(src, split1, AB, CD, nv, d, lo, hi, G):
    """ab_cd_split (sr_kernels.cuh): G lanes, each round's bounded searches
    anchored by the counts the lanes next to the previous answer found."""
    j0 = lo // nv
    ab = [j0 * nv, _pair_count_at_tile(split1, AB, nv, j0), min((j0 + 1) * nv, AB[4]),
          _pair_count_at_tile(split1, AB, nv, j0 + 1)]
    cd = [max(d - (j0 + 1) * nv, 0), _pair_count_at_tile(split1, CD, nv, d // nv - j0 - 1),
          min(d - j0 * nv, CD[4]), _pair_count_at_tile(split1, CD, nv, d // nv - j0)]
    assert hi <= ab[2] or hi == lo
    while hi > lo:
        step = (hi - lo + G) // (G + 1)
        bs, s1s, s2s = [], [], []
        for j in range(G):
            m = lo + (j + 1) * step - 1
            b, s1, s2 = False, 0, 0
            if m < hi:
                x1, x2 = m + 1, d - m
                s1 = _pair_count(src, AB, ab, x1)
                s2 = _pair_count(src, CD, cd, x2)
                a = src[AB[0] + s1 - 1] if s1 > 0 else None
                if x1 - 1 - s1 >= 0:
                    y = src[AB[1] + x1 - 1 - s1]
                    a = y if a is None or a < y else a
                c = src[CD[0] + s2 - 1] if s2 > 0 else None
                if x2 - 1 - s2 >= 0:
                    y = src[CD[1] + x2 - 1 - s2]
                    c = y if c is None or c < y else c
                assert a.v == _pair_key(src, split1, AB, nv, m).v
                assert c.v == _pair_key(src, split1, CD, nv, d - 1 - m).v
                b = not (c < a)
            bs.append(b)
            s1s.append(s1)
            s2s.append(s2)
        cnt = sum(bs)
        assert bs == [True] * cnt + [False] * (G - cnt)
        mlo = lo + cnt * step - 1
        mhi = lo + (cnt + 1) * step - 1
        if cnt > 0:
            ab[0], ab[1] = mlo + 1, s1s[cnt - 1]
            cd[2], cd[3] = d - mlo, s2s[cnt - 1]
        if cnt < G and mhi < hi:
            ab[2], ab[3] = mhi + 1, s1s[cnt]
            cd[0], cd[1] = d - mhi, s2s[cnt]
        nhi = hi if cnt == G else mhi
        lo = lo + cnt * step
        hi = min(hi, nhi)
    return lo, _pair_count(src, AB, ab, lo), _pair_count(src, CD, cd, d - lo)


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


def _runs_input(rng, n, ts):
    """Keys with presorted stretches of every kind: sorted runs of random
    lengths (not aligned to tiles), reversed runs, random stretches, few
    distinct values."""
    out = []
    while len(out) < n:
        kind = rng.choice(["asc", "desc", "rand", "few"])
        ln = rng.randint(1, 6 * ts)
        if kind == "asc":
            base = rng.randrange(10 ** 6)
            out.extend(sorted(base + rng.randrange(5000) for _ in range(ln)))
        elif kind == "desc":
            out.extend(sorted((rng.randrange(10 ** 6) for _ in range(ln)), reverse=True))
        elif kind == "rand":
            out.extend(rng.randrange(10 ** 6) for _ in range(ln))
        else:
            out.extend(rng.randrange(3) for _ in range(ln))
    return out[:n]


@pytest.mark.parametrize("seed", range(8))
def test_run_steps_model(seed):
    """Block-sorted tiles merged by the run planner's steps (sr_plain.cuh):
    natural runs of whole tiles (k_runs), then steps of fan-in 2 (k_partition
    + k_merge) or 4 (k_partition, k_partition4 + k_merge4) over groups of
    consecutive runs.  Every read inside its run window or the shared buffer,
    every output tile equal to the stable merge of its group (ties: runs in
    order, then position), the step count ceil(log_f(runs)), and the result
    sorted and stable."""
    rng = random.Random(100 + seed)
    NT, IPT = 8, 3
    nv = NT * IPT
    ts = 2 * nv
    for trial in range(10):
        fan = 2 if (seed + trial) % 2 else 4
        n = rng.choice([rng.randint(1, 10 * ts), rng.randint(10 * ts, 70 * ts)])
        if trial % 3 == 0:
            vals = [rng.randrange(rng.choice([3, 10 ** 6])) for _ in range(n)]
        elif trial % 3 == 1:
            vals = _runs_input(rng, n, ts)
        else:                                      # teeth: a few long sorted runs (not tile-aligned)
            k = rng.randint(1, 9)
            vals = [i % (n // k + 1) for i in range(n)]
        
        tiles = (n + ts - 1) // ts
        keys = []
        for t in range(tiles):
            idx = sorted(range(t * ts, min(n, (t + 1) * ts)), key=lambda i: (vals[i], i))
            keys.extend(_K(vals[i], 0, i) for i in idx)
        lo_ = [keys[t * ts].v for t in range(tiles)]
        hi_ = [keys[min(n, (t + 1) * ts) - 1].v for t in range(tiles)]
        rs0, nruns, nsteps = _runs(lo_, hi_, tiles, fan)
        levels = 0
        while (1 << levels) < tiles:
            levels += 1
        max_steps = levels if fan == 2 else (levels + 1) // 2
        assert nsteps <= max_steps
        mt = (n + nv - 1) // nv
        span = 1
        for step in range(nsteps):
            split1 = [_partition2(keys, n, ts, tiles, nv, rs0, nruns, span, b) for b in range(mt + 1)]
            new = []
            if fan == 2:
                for b in range(mt):
                    out0, out1 = b * nv, min(b * nv + nv, n)
                    a0, a_beg, a_end, b_end = split1[b]
                    a1 = a_end if out1 == b_end else split1[b + 1][0]
                    b0 = a_end + (out0 - a_beg) - (a0 - a_beg)
                    cnt = out1 - out0
                    assert a_beg <= a0 <= a1 <= a_end and a_end <= b0 <= b0 + cnt - (a1 - a0) <= b_end
                    A = [_K(k.v, 0, k.pos) for k in keys[a0:a1]]
                    B = [_K(k.v, 1, k.pos) for k in keys[b0:b0 + cnt - (a1 - a0)]]
                    got = sorted(A + B, key=lambda k: (k.v, k.run, k.pos))
                    grp = sorted(([_K(k.v, 0, k.pos) for k in keys[a_beg:a_end]] +
                                  [_K(k.v, 1, k.pos) for k in keys[a_end:b_end]]),
                                 key=lambda k: (k.v, k.run, k.pos))
                    assert [k.full() for k in got] == [k.full() for k in grp[out0 - a_beg:out1 - a_beg]]
                    new.extend(_K(k.v, 0, k.pos) for k in got)
            else:
                G = rng.choice([1, 2, 4, 8])
                split4 = [_partition4(keys, n, ts, tiles, nv, rs0, nruns, span, split1, b, G) for b in range(mt + 1)]
                for b in range(mt):
                    out0, out1 = b * nv, min(b * nv + nv, n)
                    beg, ends = split4[b][:4], split4[b][4:]
                    last = out1 == ends[3]
                    end = ends if last else split4[b + 1][:4]
                    ln = [end[i] - beg[i] for i in range(4)]
                    assert sum(ln) == out1 - out0 and min(ln) >= 0
                    # each key of the group tagged with its run, for the tie order
                    q = _nrun_of(rs0, nruns, tiles, out0 // ts)
                    g0 = (q // (4 * span)) * (4 * span)
                    e5 = [_nrun_pos(rs0, nruns, g0 + i * span, ts, n) for i in range(5)]
                    assert e5[1:] == ends
                    tg = [None] * n
                    for r in range(4):
                        for g in range(e5[r], e5[r + 1]):
                            tg[g] = _K(keys[g].v, r, keys[g].pos)
                    got = _merge_tile4(tg, n, out0, out1 - out0, beg, ln, NT, IPT, bulk=(b + trial) % 2 == 0)
                    grp = sorted(k.full() for k in tg[e5[0]:e5[4]])
                    assert [k.full() for k in got] == grp[out0 - e5[0]:out1 - e5[0]], (n, b)
                    new.extend(_K(k.v, 0, k.pos) for k in got)
            keys = new
            span *= fan
        assert [(k.v, k.pos) for k in keys] == sorted((v, i) for i, v in enumerate(vals))


@pytest.mark.parametrize("seed", range(4))
def test_neighbour_repair_model(seed):
    """k_repair_plan + k_repair (sr_kernels.cuh): when every block-sorted
    tile's keys are <= those of the tile two places on, merging in place the
    window at each tile boundary (tile t's keys above tile t+1's smallest,
    tile t+1's keys below tile t's largest) sorts the array, stably; the
    windows never overlap and stay inside their two tiles.  Inputs: k-distance
    lists (Section 2) with k up to half a tile, few distinct values, and
    windows too large (the repair then gives way to the merge steps)."""
    rng = random.Random(300 + seed)
    ts, cap = 48, 24
    tried = applied = 0
    for trial in range(60):
        n = rng.randint(3 * ts, 40 * ts)
        k = rng.choice([1, 3, 8, ts // 2, ts])
        vals = list(range(n))
        for s0 in range(0, n, k + 1):                 # k-distance: sections of k+1 shuffled
            sec = vals[s0:s0 + k + 1]
            rng.shuffle(sec)
            vals[s0:s0 + k + 1] = sec
        if trial % 5 == 4:
            vals = [v // 7 for v in vals]             # repeated values
        tiles = (n + ts - 1) // ts
        keys = []
        for t in range(tiles):
            idx = sorted(range(t * ts, min(n, (t + 1) * ts)), key=lambda i: (vals[i], i))
            keys.extend(_K(vals[i], 0, i) for i in idx)
        lo_ = [keys[t * ts].v for t in range(tiles)]
        hi_ = [keys[min(n, (t + 1) * ts) - 1].v for t in range(tiles)]
        far = any(hi_[q] > lo_[q + 2] for q in range(tiles - 2))
        _, nruns, steps = _runs(lo_, hi_, tiles, 2)
        if far or steps == 0:
            continue
        tried += 1
        src = _Checked(keys, "keys")
        win, fail, covered = [], False, set()
        for t in range(tiles - 1):                    # k_repair_plan
            x0, x1, y0, y1 = t * ts, t * ts + ts, t * ts + ts, min(t * ts + 2 * ts, n)
            a, b = x0, x1
            while a < b:
                m = (a + b) >> 1
                if src[m].v <= lo_[t + 1]:
                    a = m + 1
                else:
                    b = m
            e, f = y0, y1
            while e < f:
                m = (e + f) >> 1
                if src[m].v < hi_[t]:
                    e = m + 1
                else:
                    f = m
            na, nb = x1 - a, e - y0
            if na + nb > cap:
                fail = True
            win.append((na, nb))
        if fail:
            continue
        applied += 1
        out = list(keys)
        for t, (na, nb) in enumerate(win):            # k_repair: merge_tile in place
            if na == 0 or nb == 0:
                continue
            mid = (t + 1) * ts
            rng_ = set(range(mid - na, mid + nb))
            assert not (rng_ & covered)                # windows never overlap
            covered |= rng_
            A = [_K(k.v, 0, k.pos) for k in keys[mid - na:mid]]
            B = [_K(k.v, 1, k.pos) for k in keys[mid:mid + nb]]
            merged = sorted(A + B, key=lambda k: (k.v, k.run, k.pos))
            out[mid - na:mid + nb] = [_K(k.v, 0, k.pos) for k in merged]
        assert [(k.v, k.pos) for k in out] == sorted((v, i) for i, v in enumerate(vals)), (n, k)
    assert tried >= 20 and applied >= 10, (tried, applied)


def _tile_order(tmin, tmax, n, ts, tiles, strict, NT):
    """k_tile_order with NT threads: chunked running max forward (each tile's
    chain start), running min backward (its chain end); dest = first + last - q."""
    full = n // ts

    def desc(q):
        if q <= 0 or q >= full:
            return False
        down = tmax[q] < tmin[q - 1] if strict else tmax[q] <= tmin[q - 1]
        return down and not (tmax[q - 1] <= tmin[q])

    dest = [0] * tiles
    carry = 0
    for t0 in range(0, tiles, NT):
        run = carry
        for t in range(NT):
            q = t0 + t
            start = q if (q < tiles and not desc(q)) else -1
            run = max(run, start)
            if q < tiles:
                dest[q] = run
        carry = run
    carry, any_ = tiles - 1, False
    t1 = tiles
    while t1 > 0:
        run = carry
        for t in reversed(range(NT)):
            q = t1 - NT + t
            end = q if (0 <= q < tiles and not desc(q + 1)) else 10 ** 9
            run = min(run, end)
            if 0 <= q < tiles:
                first = dest[q]

                def asc(x, y):
                    return 1 if (x >= 0 and y < tiles and tmax[x] <= tmin[y]) else 0
                gain = (run - first) + asc(first - 1, run) + asc(first, run + 1) - asc(first - 1, first) - \
                    asc(run, run + 1)
                flip = run > first and gain > 0
                any_ |= flip
                dest[q] = first + run - q if flip else q
        carry = run
        t1 -= NT
    return dest, any_, desc


@pytest.mark.parametrize("strict", [False, True])
def test_tile_order_model(strict):
    """Chains of tiles in descending order reversed by the block sort: dest is
    a permutation that reverses every maximal chain of full tiles whose
    boundaries descend (strictly, for stable pair sorts) and fixes every other
    tile; after it the chain's tiles ascend.  Against a direct search of the
    chains, with chunks of a few threads so the scans' carries are used."""
    rng = random.Random(7 + strict)
    for trial in range(300):
        ts = rng.choice([1, 3, 8])
        tiles = rng.randint(1, 40)
        n = tiles * ts - (rng.randint(0, ts - 1) if rng.random() < 0.5 else 0)
        tiles = (n + ts - 1) // ts
        if tiles == 0:
            continue
        # tile extremes from a random sequence of ascending / descending stretches
        lo_, hi_ = [], []
        v = 1000
        for t in range(tiles):
            step = rng.choice([-40, -40, 40, 0, 5])
            v += step
            w = rng.choice([0, 3, 10])
            lo_.append(v)
            hi_.append(v + w)
        dest, any_, desc = _tile_order(lo_, hi_, n, ts, tiles, strict, rng.choice([1, 2, 4, 8]))
        assert sorted(dest) == list(range(tiles))
        # direct: maximal chains [a, b] of descending boundaries, turned when
        # that lowers the number of natural runs (counted on the result)
        def runs_of(order):
            return 1 + sum(1 for i in range(1, len(order)) if hi_[order[i - 1]] > lo_[order[i]])
        want = list(range(tiles))
        q = 0
        while q < tiles:
            b = q
            while b + 1 < tiles and desc(b + 1):
                b += 1
            trial_order = list(range(tiles))
            trial_order[q:b + 1] = reversed(trial_order[q:b + 1])
            if b > q and runs_of(trial_order) < runs_of(list(range(tiles))):
                for r in range(q, b + 1):
                    want[r] = q + b - r
            q = b + 1
        assert dest == want
        assert any_ == (want != list(range(tiles)))
        order = [None] * tiles
        for q in range(tiles):
            order[dest[q]] = q
        assert runs_of(order) <= runs_of(list(range(tiles)))
        for q in range(tiles):
            if dest[q] != q:
                assert (q + 1) * ts <= n                # only full tiles move
        # moved chains ascend (each tile's keys <= the next's; strictly for strict)
        pos = [None] * tiles
        for q in range(tiles):
            pos[dest[q]] = q
        for p in range(1, tiles):
            a, b = pos[p - 1], pos[p]
            if dest[a] != a and dest[b] != b and abs(a - b) == 1:
                assert hi_[a] <= lo_[b] and (not strict or hi_[a] < lo_[b])


def test_few_keys_model():
    """k_few_sample's bitonic network over the sampled set (padded to a power
    of two with the largest image) sorts any k <= 4,096 images; k_few_write's
    exclusive scan (16 counts per thread, 8 partial sums per lane of one warp)
    and its search for each output's key write every key count times, in
    order."""
    rng = random.Random(11)
    for k in (1, 2, 3, 16, 17, 100, 1000, 4095, 4096):
        v = [rng.randrange(1 << 32) for _ in range(k)]
        P = 1
        while P < k:
            P <<= 1
        s = v + [0xFFFFFFFF] * (P - k)
        size = 2
        while size <= P:
            stride = size >> 1
            while stride > 0:
                for q in range(P // 2):
                    lo = 2 * stride * (q // stride) + (q % stride)
                    hi = lo + stride
                    assert hi < P
                    up = (lo & size) == 0
                    if (s[lo] > s[hi]) == up:
                        s[lo], s[hi] = s[hi], s[lo]
                stride >>= 1
            size <<= 1
        assert s[:k] == sorted(v)
        # scan of the counts as k_few_write does it
        counts = [rng.randint(0, 5) for _ in range(k)]
        PER = 4096 // 256
        part = [sum(counts[q] for q in range(t * PER, t * PER + PER) if q < k) for t in range(256)]
        excl, acc = [0] * 256, 0
        for lane in range(32):                       # 8 partial sums per lane, then the warp scan
            for w in range(8):
                excl[lane * 8 + w] = acc
                acc += part[lane * 8 + w]
        start = []
        for t in range(256):
            run = excl[t]
            for e in range(PER):
                q = t * PER + e
                if q < k:
                    start.append(run)
                    run += counts[q]
        assert start == [sum(counts[:q]) for q in range(k)]
        n = sum(counts)
        out = []
        for i in range(n):                           # which(i): the last q < k with start[q] <= i
            lo, hi = 0, k - 1
            while lo < hi:
                mid = (lo + hi + 1) >> 1
                if start[mid] <= i:
                    lo = mid
                else:
                    hi = mid - 1
            out.append(s[lo])
        assert out == [s[q] for q in range(k) for _ in range(counts[q])]


def test_few_keys_chunked_write_and_lookup_model():
    """k_few_write's warp chunks (lane l writes 16-byte groups l, l+32, ... of
    each 256-group chunk, one search per lane per chunk, then a key index that
    only moves forward) write every position exactly once with the right key,
    whatever the grid; k_few_count's hash table maps every image of the set to
    its rank and reports a key outside the set."""
    rng = random.Random(12)
    for trial in range(30):
        k = rng.choice([1, 2, 5, 64, 300, 4096])
        counts = [rng.choice([0, 1, 3, 9, 1000]) for _ in range(k)]
        counts[rng.randrange(k)] += 1
        n = sum(counts)
        start, acc = [], 0
        for c in counts:
            start.append(acc)
            acc += c
        want = [q for q in range(k) for _ in range(counts[q])]

        def which(i):
            lo, hi = 0, k - 1
            while lo < hi:
                mid = (lo + hi + 1) >> 1
                if start[mid] <= i:
                    lo = mid
                else:
                    hi = mid - 1
            return lo
        nv = n // 4
        out = [None] * n
        blocks, warps_per = rng.choice([1, 3, 7]), 8
        warps = blocks * warps_per
        CH = 32 * 8
        for wid in range(warps):
            c0 = wid * CH
            while c0 < nv:
                end = min(c0 + CH, nv)
                for lane in range(32):
                    v = c0 + lane
                    if v >= end:
                        continue
                    j = which(4 * v)
                    ej = start[j + 1] if j + 1 < k else float("inf")   # where run j ends
                    while v < end:
                        i = 4 * v
                        if i + 4 <= ej:                 # the whole vector in run j
                            for m in range(4):
                                assert out[i + m] is None
                                out[i + m] = j
                            v += 32
                            continue
                        for m in range(4):
                            while j + 1 < k and start[j + 1] <= i + m:
                                j += 1
                            assert out[i + m] is None
                            out[i + m] = j
                        ej = start[j + 1] if j + 1 < k else float("inf")
                        v += 32
                c0 += warps * CH
        for i in range(4 * nv, n):                   # the scalar tail
            out[i] = which(i)
        assert out == want
    # the count pass's table: image -> rank + 1, linear probing, at most half full
    imgs = sorted(rng.sample(range(1 << 32), 4096))
    SL, tab = 1 << 13, [0] * (1 << 13)
    for q, u in enumerate(imgs):
        h = (u * 2654435761 % (1 << 32)) >> (32 - 13)
        while tab[h]:
            h = (h + 1) & (SL - 1)
        tab[h] = (u << 32) | (q + 1)

    def look(u):
        h = (u * 2654435761 % (1 << 32)) >> (32 - 13)
        for _ in range(SL):
            e = tab[h]
            if e == 0:
                return None
            if e >> 32 == u:
                return (e & 0xFFFFFFFF) - 1
            h = (h + 1) & (SL - 1)
        return None
    assert all(look(u) == q for q, u in enumerate(imgs))
    s = set(imgs)
    for _ in range(2000):
        u = rng.randrange(1 << 32)
        assert look(u) == (imgs.index(u) if u in s else None)


def _marked_keys_step(rd, a, b, IPT, lt):
    """serial_merge_marked_keys (sr_device.cuh): the heads kept as (the head
    not taken, its index) and (the key just loaded, its index); a step takes
    the smaller head and moves only the taken side's index."""
    x, px = rd(a), a
    y, py = rd(b), b
    out = []
    for _ in range(IPT):
        p = lt(y, x)
        out.append(y if p else x)
        o, po = (x, px) if p else (y, py)
        pt = (py if p else px) + 1
        x, px = o, po
        y, py = rd(pt), pt
    return out


def test_marked_merge_tile_model():
    """merge_tile's bulk staging (sr_kernels.cuh) with end-marked windows: A's
    4-key groups, a spare group, B's groups, umax after each window, and the
    one-comparison merge step (serial_merge_marked).  Outputs equal the stable
    merge (ties to A), every staged slot fits merge_tile_sv, and every read
    stays below it plus the IPT + 8 keys of slack."""
    rng = random.Random(11)
    UMAX = 10 ** 9
    for trial in range(400):
        NT, IPT = rng.choice([(4, 3), (8, 5), (16, 7), (8, 25)])
        NV = NT * IPT
        SV = NV + 20
        size = SV + IPT + 8
        cnt = rng.randint(1, NV)
        acnt = rng.randint(0, cnt)
        bcnt = cnt - acnt
        alpha = rng.choice([3, 50, 10 ** 6])
        A = sorted(rng.randrange(alpha) for _ in range(acnt))
        B = sorted(rng.randrange(alpha) for _ in range(bcnt))
        a0, b0 = rng.randint(0, 50), rng.randint(0, 50)
        g0a, g0b = a0 & ~3, b0 & ~3
        nag = (((a0 + acnt + 3) & ~3) - g0a) >> 2 if acnt else 0
        nbg = (((b0 + bcnt + 3) & ~3) - g0b) >> 2 if bcnt else 0
        sa = a0 - g0a
        sb = 4 * (nag + 1) + (b0 - g0b)
        assert 4 * (nag + 1 + nbg) <= NV + 16 and sb + bcnt < SV
        # garbage: compared only by the steps of outputs past cnt, never output
        smem = [(rng.randrange(2 * alpha), 8, i) for i in range(size)]
        for i, v in enumerate(A):
            smem[sa + i] = (v, 0, i)
        for i, v in enumerate(B):
            smem[sb + i] = (v, 1, i)
        smem[sa + acnt] = (UMAX, 9, 0)
        smem[sb + bcnt] = (UMAX, 9, 1)
        reads = [0]

        def rd(i):
            assert 0 <= i < size
            reads[0] = max(reads[0], i)
            return smem[i]

        def lt(x, y):                                 # the order of the images alone
            return x[0] < y[0]
        out = []
        for t in range(NT):
            diag = min(t * IPT, cnt)
            lo, hi = max(0, diag - bcnt), min(diag, acnt)
            while lo < hi:
                m = (lo + hi) >> 1
                if not lt(rd(sb + diag - 1 - m), rd(sa + m)):
                    lo = m + 1
                else:
                    hi = m
            a, b = sa + lo, sb + diag - lo
            ak, bk = rd(a), rd(b)
            k = []
            for i in range(IPT):
                take_a = not lt(bk, ak)
                k.append(ak if take_a else bk)
                nx = (a if take_a else b) + 1
                nk = rd(nx)
                if take_a:
                    a, ak = nx, nk
                else:
                    b, bk = nx, nk
            out.extend(k[:max(0, min(IPT, cnt - diag))])
        want = sorted([(v, 0, i) for i, v in enumerate(A)] + [(v, 1, i) for i, v in enumerate(B)])
        assert out == want, (NT, IPT, acnt, bcnt)
        assert reads[0] < size


def _block_sort_pp(keys, NT, IPT, umax, keys_only=False):
    """block_sort_pp and block_sort_rs (sr_device.cuh) on one tile of NT*IPT
    keys: the per-warp stretches of the warp-synchronised rounds and the end
    marks (the layout both share; block_sort_rs reads a round's runs from the
    buffer it then writes, after its warp or block has read them all).  Checks
    every read against the buffer and, in those rounds, every read and write
    against the warp's own stretch, and that a round reads only slots the
    round before it wrote.  keys_only: block_sort_rs for keys alone, whose
    marked rounds take serial_merge_marked_keys's step."""
    W = 32 * IPT + 32
    size = NT * IPT + NT
    assert (NT // 32) * W == size
    bufs = [[None] * size, [None] * size]
    regs = [sorted(keys[t * IPT:(t + 1) * IPT]) for t in range(NT)]
    fast = not any(getattr(r[-1], "v", r[-1]) == getattr(umax, "v", umax) for r in regs)
    for t in range(NT):
        w, lane = t >> 5, t & 31
        for i in range(IPT):
            bufs[0][w * W + lane * (IPT + 1) + i] = regs[t][i]
        bufs[0][w * W + lane * (IPT + 1) + IPT] = umax
    src, dst = 0, 1
    coop = 2
    while coop <= NT:
        new = [None] * size
        for t in range(NT):
            w = t >> 5
            first = t & ~(coop - 1)
            run = (coop >> 1) * IPT
            diag = (t - first) * IPT
            if coop <= 32:
                gl = (first & 31) // coop
                a0 = w * W + 2 * gl * (run + 1)
                b0 = a0 + run + 1
                o0 = w * W + gl * (2 * run + 1)
                lo_ok, hi_ok = w * W, (w + 1) * W
            else:
                rs = (coop // 64) * W
                g = first // coop
                a0, o0 = 2 * g * rs, 2 * g * rs
                b0 = a0 + rs
                lo_ok, hi_ok = 0, size

            def rd(i):
                assert lo_ok <= i < hi_ok and bufs[src][i] is not None, (coop, t, i)
                return bufs[src][i]
            lo, hi = max(0, diag - run), min(diag, run)
            while lo < hi:
                mid = (lo + hi) >> 1
                if not (rd(b0 + diag - 1 - mid) < rd(a0 + mid)):
                    lo = mid + 1
                else:
                    hi = mid
            a, b, a_end, b_end = a0 + lo, b0 + diag - lo, a0 + run, b0 + run
            if fast and keys_only:
                def rd_run(i):                        # inside the two runs and their marks
                    assert a0 <= i <= a_end or b0 <= i <= b_end, (coop, t, i)
                    return rd(i)
                for i, v in enumerate(_marked_keys_step(rd_run, a, b, IPT, lambda x, y: x < y)):
                    o = o0 + diag + i
                    assert lo_ok <= o < hi_ok
                    new[o] = v
                if t - first == coop - 1:
                    assert lo_ok <= o0 + 2 * run < hi_ok
                    new[o0 + 2 * run] = umax
                continue
            ak, bk = rd(a), rd(b)
            for i in range(IPT):
                tb = (bk < ak) if fast else (b < b_end and (a >= a_end or bk < ak))
                o = o0 + diag + i
                assert lo_ok <= o < hi_ok
                new[o] = bk if tb else ak
                nx = (b if tb else a) + 1
                nk = rd(nx)
                if tb:
                    b, bk = nx, nk
                else:
                    a, ak = nx, nk
            if t - first == coop - 1:
                assert lo_ok <= o0 + 2 * run < hi_ok
                new[o0 + 2 * run] = umax
        bufs[dst] = new
        src, dst = dst, src
        coop <<= 1
    return bufs[src][:NT * IPT]


@pytest.mark.parametrize("NT,IPT", [(64, 3), (128, 5), (256, 3)])
def test_block_sort_pp_model(NT, IPT):
    """The ping-pong block sort's layout: sorted tiles with and without keys
    equal to the end mark (the bounded rounds), every access in bounds and in
    the accessing warp's stretch while warps synchronise alone."""
    rng = random.Random(NT + IPT)
    umax = 2 ** 32 - 1
    for trial in range(6):
        n = NT * IPT
        if trial % 3 == 0:
            keys = [rng.randrange(2 ** 32 - 1) for _ in range(n)]
        elif trial % 3 == 1:
            keys = [rng.randrange(7) for _ in range(n)]
        else:
            keys = [rng.choice([0, umax, rng.randrange(100)]) for _ in range(n)]
        assert _block_sort_pp(keys, NT, IPT, umax) == sorted(keys)
        assert _block_sort_pp(keys, NT, IPT, umax, keys_only=True) == sorted(keys)


def test_block_sort_rs_payload_model():
    """block_sort_rs with payloads: keys that compare by value alone and carry
    their tile position; ties must keep that order (the stable tile sort), with
    and without keys equal to the end mark."""
    rng = random.Random(5)
    umax = 2 ** 32 - 1
    NT, IPT = 64, 5
    for trial in range(8):
        n = NT * IPT
        vals = [rng.choice([rng.randrange(4), umax] if trial % 2 else [rng.randrange(4)]) for _ in range(n)]
        keys = [_K(v, 0, i) for i, v in enumerate(vals)]
        out = _block_sort_pp(keys, NT, IPT, _K(umax, 9, -1))
        assert [k.full() for k in out] == sorted(k.full() for k in keys)
