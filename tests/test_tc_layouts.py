"""Shared-memory layouts of the mma.sync split-precision tensor-core passes
(host-side design check, no GPU).  These passes serve lines of 16 and 32
points; longer lines run on tcgen05, whose operand layout is fixed by the
hardware descriptors (fft_tc5.cuh) and whose results are checked on the GPU.

The mma.sync passes store a tile between passes with an XOR swizzle: element
(row e, column c) sits at row e ^ P(e), column c ^ H(e), each bit of H and P
the parity of a set of row bits.  The masks below restate TcSwz of
fft_tc.cuh.  For every tile shape these passes launch, this test enumerates
the shared-memory accesses of every pass with the kernels' lane-to-element
mapping.  It checks that each layout is a bijection and that the swizzled
accesses need one wavefront per half-warp (64-bit accesses: 16 distinct
8-byte bank slots).  Only the first radix-8 stage, which reads the plain
layout written by the TMA, is allowed 4-way conflicts.  The numerical
results of the same passes are checked on the GPU against the oracle
(tests/test_gpu_parity.py, -k mixed).
"""

from collections import Counter

import pytest


def par(mask, r):
    return bin(mask & r).count("1") & 1


def xor_layout(cx, hmasks, pmask):
    def phys(r, c):
        h = 0
        for k, m in enumerate(hmasks):
            h |= par(m, r) << k
        return (r ^ par(pmask, r)) * cx + (c ^ h)
    return phys


def plain(cx):
    return lambda r, c: r * cx + c


def bits(*bs):
    m = 0
    for b in bs:
        m |= 1 << b
    return m


def tc_swz(logn, cx):
    """TcSwz: A = bits {0,3,6,9}, C = bits {1,4,7,10} (+ bit Q+1 when C holds
    neither Q nor Q+1), B = bit Q or Q+1, Q = log2 N - 2."""
    q = logn - 2
    a, c0 = 0x249, 0x492
    c = c0 if (c0 >> q) & 3 else c0 | (1 << (q + 1))
    b = (1 << q) if (c >> (q + 1)) & 1 else (1 << (q + 1))
    if cx == 16:
        return xor_layout(cx, [a, 0, b, c], 0)
    return xor_layout(cx, [a, 0, b], c)


def shape(logn, is_y):
    """Tile of the mma.sync form: values per thread E, threads per line TL,
    columns CX, threads (the TShape rule for 16- and 32-point lines)."""
    n = 1 << logn
    e = 8
    tl = n // e
    cx = min(16, 512 // tl)
    return n, e, tl, cx, cx * tl


def wavefronts(accesses, phys):
    """Most accesses one 8-byte bank slot receives within a half-warp."""
    worst = 0
    for h in (0, 16):
        cnt = Counter(phys(r, c) % 16 for r, c in accesses[h:h + 16])
        worst = max(worst, max(cnt.values()))
    return worst


def stage8_accesses(n, cx, threads, ns):
    """(reads, writes) of one tensor-core radix-8 stage of stride ns: lane
    (g, t) reads inputs 2t, 2t+1 of B column g and writes output g of B
    columns 2t, 2t+1; B column beta = 8 (w GROUPS + G) + n."""
    warps = threads // 32
    groups = cx * n // 8 // (8 * warps)
    reads, writes = [], []
    for w in range(warps):
        for gg in range(groups):
            base8 = (w * groups + gg) * 8
            for d in (0, 1):
                acc = []
                for lane in range(32):
                    g, t = lane >> 2, lane & 3
                    beta = base8 + g
                    acc.append((beta // cx + (2 * t + d) * (n // 8), beta % cx))
                reads.append(acc)
            for i in (0, 1):
                acc = []
                for lane in range(32):
                    g, t = lane >> 2, lane & 3
                    beta = base8 + 2 * t + i
                    b = beta // cx
                    acc.append(((b // ns) * ns * 8 + b % ns + g * ns, beta % cx))
                writes.append(acc)
    return reads, writes


def f32_accesses(n, cx, threads, rp, ns):
    """(reads, writes) of the float32 radix-rp last stage (one butterfly per thread and round)."""
    nbf = cx * n // rp
    reads, writes = [], []
    for q in range((nbf + threads - 1) // threads):
        for w in range(threads // 32):
            for r in range(rp):
                ra, wa = [], []
                for lane in range(32):
                    beta = 32 * w + lane + q * threads
                    c, b = beta % cx, beta // cx
                    ra.append((b + r * (n // rp), c))
                    wa.append(((b // ns) * ns * rp + b % ns + r * ns, c))
                reads.append(ra)
                writes.append(wa)
    return reads, writes


def copy_accesses(n, cx, threads, e):
    """The kernel's copy-out of the result (and the inverse pass's copy-in):
    thread (c = tid % CX, j = tid / CX) takes rows j + TL m of column c."""
    tl = n // e
    out = []
    for w in range(threads // 32):
        for m in range(e):
            out.append([((32 * w + lane) // cx + tl * m, (32 * w + lane) % cx) for lane in range(32)])
    return out


def bijective(phys, n, cx):
    s = {phys(r, c) for r in range(n) for c in range(cx)}
    return len(s) == n * cx and min(s) == 0 and max(s) == n * cx - 1


CASES = [(logn, is_y) for logn in (4, 5) for is_y in (True, False)]


@pytest.mark.parametrize("logn,is_y", CASES)
def test_tensor_core_layouts(logn, is_y):
    n, e, tl, cx, threads = shape(logn, is_y)
    assert cx in (8, 16) and threads <= 512
    worst = {}

    def note(kind, accesses, phys):
        worst[kind] = max(worst.get(kind, 0), max(wavefronts(a, phys) for a in accesses))

    p = plain(cx)
    if True:
        sw = tc_swz(logn, cx)
        assert bijective(sw, n, cx)
        ns = 1
        while n // ns >= 8:
            r, w = stage8_accesses(n, cx, threads, ns)
            note("first stage reads (plain)" if ns == 1 else "swizzled", r, p if ns == 1 else sw)
            note("swizzled" if ns * 8 < n else "plain writes", w, sw if ns * 8 < n else p)
            ns *= 8
        rem = n // ns
        if rem > 1:
            r, w = f32_accesses(n, cx, threads, 4 if rem >= 4 else 2, ns)
            note("swizzled", r, sw)
            note("plain writes", w, p)
        note("copies (plain)", copy_accesses(n, cx, threads, e), p)
    assert worst["swizzled"] == 1, worst
    assert worst["first stage reads (plain)"] <= 4, worst
    assert worst["copies (plain)"] == 1, worst
    assert worst.get("plain writes", 1) == 1, worst
