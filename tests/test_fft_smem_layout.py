"""Shared-memory bank model of the register FFT engine (fft_kernels.cu,
lengths 64-1024): every warp instruction of every pass of one CTA, split into
half-warps of 8-byte words (one 128-byte wavefront each when free of
conflicts), counted against 32 four-byte banks.

Pins the layout choices the kernels rely on: the exchange index
l ^ ((l >> 3) & 15) with team rows N + 16/NT apart, and the pass-major
twiddle table (pass s: w^(j k) at offset + (j - 1) P + k), are conflict-free
for every length and every team count the library launches; indexing one
length-N table by j k N / (P R) is not."""
import pytest


def ilog2(n):
    return n.bit_length() - 1


def radices(n):
    lg = ilog2(n)
    return [8] * (lg // 3) + ([1 << (lg % 3)] if lg % 3 else [])


def xswz(l):
    return l ^ ((l >> 3) & 15)


def wavefronts(addrs):
    """(wavefronts, conflict-free wavefronts) of one warp access of 8-byte
    words at float2 indices (CTAs smaller than a warp fill part of one)."""
    total = ideal = 0
    for half in (addrs[:16], addrs[16:]):
        if not half:
            continue
        banks = {}
        for a in half:
            for word in (2 * a, 2 * a + 1):
                banks.setdefault(word % 32, set()).add(word)
        total += max(len(v) for v in banks.values())
        ideal += 1
    return total, ideal


def warps(threads):
    for w0 in range(0, threads, 32):
        yield range(w0, min(w0 + 32, threads))


def exchange_ratio(n, nt):
    """Wavefronts of the exchanges (writes of pass s, reads of pass s+1) over
    the conflict-free count."""
    tt, ldx = n // 8, n + 16 // nt
    actual = ideal = 0
    p = 1
    rs = radices(n)
    for s, r in enumerate(rs[:-1]):
        for q in range(8 // r):
            for m in range(r):
                for lanes in warps(tt * nt):
                    ad = []
                    for t in lanes:
                        i, team = t // nt, t % nt
                        b = i + q * tt
                        k = b & (p - 1)
                        ad.append(team * ldx + xswz((b - k) * r + k + m * p))
                    wf, wf0 = wavefronts(ad)
                    actual += wf
                    ideal += wf0
        for e in range(8):
            for lanes in warps(tt * nt):
                wf, wf0 = wavefronts([(t % nt) * ldx + xswz(t // nt + tt * e) for t in lanes])
                actual += wf
                ideal += wf0
        p *= r
    return actual / ideal if ideal else 1.0


def twiddle_ratio(n, nt, pass_major):
    tt = n // 8
    actual = ideal = 0
    p, off = 1, 0
    for r in radices(n):
        if p > 1:
            for q in range(8 // r):
                for j in range(1, r):
                    for lanes in warps(tt * nt):
                        ad = []
                        for t in lanes:
                            k = (t // nt + q * tt) & (p - 1)
                            ad.append(off + (j - 1) * p + k if pass_major else j * k * (n // (p * r)))
                        wf, wf0 = wavefronts(ad)
                        actual += wf
                        ideal += wf0
            off += (r - 1) * p
        p *= r
    return actual / ideal, off


LENGTHS = [64, 128, 256, 512, 1024]


@pytest.mark.parametrize("n", LENGTHS)
@pytest.mark.parametrize("nt", [1, 2, 4, 8])
def test_exchanges_are_conflict_free(n, nt):
    assert exchange_ratio(n, nt) == 1.0


@pytest.mark.parametrize("n", LENGTHS)
@pytest.mark.parametrize("nt", [1, 2, 4, 8])
def test_pass_major_twiddles_are_conflict_free_and_fit(n, nt):
    ratio, entries = twiddle_ratio(n, nt, pass_major=True)
    assert ratio == 1.0
    assert entries <= n          # the kernels stage the table in an N-entry buffer


def test_one_table_indexed_by_stride_has_conflicts():
    ratio, _ = twiddle_ratio(1024, 4, pass_major=False)
    assert ratio > 1.5


def test_a_pitch_of_n_plus_4_conflicts_for_two_and_eight_teams():
    def ratio_with_pitch(n, nt, pad):
        tt, ldx = n // 8, n + pad
        actual = ideal = 0
        for e in range(8):
            for lanes in warps(tt * nt):
                wf, wf0 = wavefronts([(t % nt) * ldx + xswz(t // nt + tt * e) for t in lanes])
                actual += wf
                ideal += wf0
        return actual / ideal
    assert ratio_with_pitch(1024, 2, 4) > 1.0 and ratio_with_pitch(1024, 8, 4) > 1.0
    assert ratio_with_pitch(1024, 2, 8) == 1.0 and ratio_with_pitch(1024, 8, 2) == 1.0


def test_closed_form_positions_equal_the_swizzle():
    """The kernels compute exchange positions as a per-thread base plus a
    compile-time offset (xpos for writes from P = 64 up, xrd for reads with
    N/8 >= 16); both are identities of the swizzled index for every length,
    pass, butterfly and element."""
    def xpos(r, p, b, k, m):
        if p >= 128:
            return (b - k) * r + (k ^ ((k >> 3) & 15)) + m * p
        if p == 64:
            return (b - k) * r + ((k ^ (k >> 3)) ^ ((m & 1) << 3)) + m * p
        return xswz((b - k) * r + k + m * p)

    def xrd(tt, i, e):
        return (i ^ (((i >> 3) + (tt // 8) * e) & 15)) + tt * e if tt >= 16 else xswz(i + tt * e)

    for n in LENGTHS:
        tt, p = n // 8, 1
        for r in radices(n):
            for i in range(tt):
                for q in range(8 // r):
                    b = i + q * tt
                    k = b & (p - 1)
                    for m in range(r):
                        assert xpos(r, p, b, k, m) == xswz((b - k) * r + k + m * p)
                for e in range(8):
                    assert xrd(tt, i, e) == xswz(i + tt * e)
            p *= r
