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
