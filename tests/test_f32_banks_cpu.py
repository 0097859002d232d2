"""Shared-memory bank model of the FP32 line operators (kernels_f32.cu) and
of the adjoint's 64-thread segment kernel for long 1D lines.

The address of every shared-memory access of k_f32_fwd / k_f32_adj is
restated here from the kernel (layouts vp, sp<Q>, the lane orders of the
zeroing and of the pencil passes, the window starts of the Geom constants)
and the accesses of each warp instruction are counted in wavefronts the way
the shared-memory unit serves them: 32 lanes at once for 4-byte accesses, 16
for 8-byte, 8 for 16-byte, one wavefront per distinct word in the busiest
bank.  Every instantiation (PM in {4, 8, 10}, Q in {2, 4}, N = 2048 / 4096)
must need no more wavefronts than its bytes demand; only the data-dependent
gather and scatter of P_Omega (Sec. 1.1) and the few edge-correction reads
are outside the model.  The GPU-side check is ncu's
l1tex__data_bank_conflicts_pipe_lsu_mem_shared counter.
"""
import pytest


def _wavefronts(addrs, width):
    lanes = {1: 32, 2: 16, 4: 8}[width]
    total = 0
    for p0 in range(0, 32, lanes):
        banks = {}
        for a in addrs[p0:p0 + lanes]:
            for w in range(width):
                banks.setdefault((a + w) % 32, set()).add(a + w)
        total += max((len(s) for s in banks.values()), default=0)
    return total


def _ideal(addrs, width):
    return -(-len(addrs) * width // 32)


def _up4(a):
    return (a + 3) // 4 * 4


def vp(k):                      # Walsh line: 4 words of padding per 16
    return k + 4 * (k >> 4)


VCH = 320                       # vp(k + 256) - vp(k)


def sp(Q, m):                   # s line
    return m ^ (((m >> 5) & 1) << 2) if Q == 2 else m


def high_pencil(c):
    hw, w = c >> 4, c >> 5
    a = (w & 3) + 8 * (w >> 2) + 4 * (hw & 1)
    return 16 * a + (c & 15)


def accesses(PM, Q, NT):
    """(site, width in words, lane addresses) of one warp instruction each."""
    N, BS = 16 * NT, 16 // Q
    BL, HS, HX = BS // 2, _up4(PM + 3), 8
    VW = 4 if BL >= 4 else 2
    OFFX = ((HX - PM // 2) % VW + VW) % VW
    NWX = (OFFX + BL + PM + VW - 1) // VW * VW
    OFFB = ((HS - PM + 1) % 4 + 4) % 4
    NWB = _up4(OFFB + BS + 2 * PM - 2)
    OFFT = (4 - (Q * (PM - 1)) % 4) % 4
    NWT = _up4(OFFT + Q * (BS + 2 * PM - 2))
    OFFA = ((HS - PM) % 4 + 4) % 4
    NWA = _up4(OFFA + 2 * BL + 2 * PM)
    VH = 256
    out = []
    for warp in range(NT // 32):
        lanes = range(32 * warp, 32 * warp + 32)
        for i in range(N // (4 * NT)):                     # adjoint: zero the line
            a = []
            for t in lanes:
                c = NT * i + t
                a.append(vp(VH + 16 * ((c & 7) + 8 * (c >> 5)) + 4 * ((c >> 3) & 3)))
            out.append(("adj zero", 4, a))
        for off, kn in ((0, "fwd"), (VH, "adj")):
            for c0 in range(0, 256, NT):                   # bits 8..: pencils at stride VCH
                act = [t for t in lanes if c0 + t < 256]
                for i in range(N // 256):
                    if act:
                        out.append((kn + " pass_high", 1, [vp(high_pencil(c0 + t) + off) + VCH * i for t in act]))
            for i in range(16):                            # bits 4-7: upper half-warp in the order i ^ 4
                a = [vp((t & 15) + 256 * (t >> 4) + off + 16 * (i ^ (4 * ((t >> 4) & 1)))) for t in lanes]
                out.append((kn + " pass_mid", 1, a))
            for r in range(0, 16, 4):                      # bits 0-3: own 16-block
                out.append((kn + " bits0_3", 4, [vp(off + 16 * t) + r for t in lanes]))
        S0 = (-(Q * (PM - 1) + OFFT)) % 16
        for w in range(0, NWT, 4):                         # adjoint T^T window
            rel = S0 + w
            out.append(("adj T^T window", 4,
                        [vp(VH + Q * BS * t - Q * (PM - 1) - OFFT - S0 + 16 * (rel >> 4)) + (rel & 15) for t in lanes]))
        for j in range(0, BS, 4):                          # s stores (forward (A), adjoint T^T)
            out.append(("s store", 4, [sp(Q, HS + BS * t + j) for t in lanes]))
        for w in range(0, NWA, 4):                         # adjoint analysis window
            out.append(("adj analysis window", 4, [sp(Q, HS + 2 * BL * t - PM - OFFA + w) for t in lanes]))
        for w in range(0, NWB, 4):                         # forward (B) T window
            out.append(("fwd T window", 4, [sp(Q, HS + BS * t - PM + 1 - OFFB + w) for t in lanes]))
        for w in range(0, NWX, VW):                        # forward (A) coefficient window (plain line)
            out.append(("fwd synthesis window", VW, [HX + BL * t - PM // 2 - OFFX + w for t in lanes]))
    return out


@pytest.mark.parametrize("PM", [4, 8, 10])
@pytest.mark.parametrize("Q", [2, 4])
@pytest.mark.parametrize("NT", [128, 256])
def test_f32_line_operators_conflict_free(PM, Q, NT):
    bad = {}
    for site, width, addrs in accesses(PM, Q, NT):
        extra = _wavefronts(addrs, width) - _ideal(addrs, width)
        if extra:
            bad[site] = bad.get(site, 0) + extra
    assert not bad, bad


def test_model_counts_conflicts():
    """The counter itself: the previous Walsh layout (16 more words per 256
    elements) conflicts in the T^T window where a quarter-warp crosses a
    256-block, and 8 lanes 32 words apart hit one bank 8 times."""
    old = lambda k: k + 4 * (k >> 4) + 16 * (k >> 8)      # noqa: E731
    a = [old(256 + 16 * t - 16) for t in range(32)]
    assert _wavefronts(a, 4) > _ideal(a, 4)
    assert _wavefronts([32 * t for t in range(8)] + [1] * 24, 1) == 8
    assert _wavefronts(list(range(32)), 1) == 1
    # the swapped half-warp visits the same pencil elements, only reordered
    for i in range(16):
        assert sorted({i ^ 4 * h for h in (0, 1)}) == sorted({i, i ^ 4})


# --- the adjoint's segment kernel for long 1D lines (k_fwht_seg64_upT) ---
def vq(k):                      # segment of 4096: 4 words of padding per 64
    return k + 4 * (k >> 6)


def seg64_accesses(PM, Q):
    """(site, width, lane addresses) of the shared-memory accesses of one
    segment: 64 threads, thread t first holds the pencil t + 64 i, then the
    64 consecutive values 64 t + r, then reads its T^T windows (Sec. 4.2)
    4 outputs at a time."""
    BO = 4096 // Q // 64
    NB = (2 * PM + 3) // 4 * 4
    OFF = ((1 - PM) * Q % 4 + 4) % 4
    CK, ST = 4, 4 * Q
    W = (OFF + Q * (CK + 2 * PM - 2) + 3) // 4 * 4
    out = []
    for warp in range(2):
        lanes = range(32 * warp, 32 * warp + 32)
        for i in range(64):                                    # pencil stores
            out.append(("seg64 pencil", 1, [vq(t + 64 * i) for t in lanes]))
        for r in range(0, 64, 4):                              # rows of 64, 16-byte vectors
            out.append(("seg64 rows", 4, [vq(64 * t + r) for t in lanes]))
        act = [t for t in lanes if BO * t >= NB and BO * t + BO <= 4096 // Q - NB]
        for c in range(BO // CK):                              # sliding T^T windows
            for w in range(0 if c == 0 else W - ST, W, 4):
                out.append(("seg64 window", 4, [vq(Q * BO * t + (1 - PM) * Q - OFF + ST * c + w) for t in act]))
    return out


@pytest.mark.parametrize("PM", [4, 8, 10])
@pytest.mark.parametrize("Q", [2, 4])
def test_seg64_layout_conflict_free(PM, Q):
    """Every access of the 64-thread segment kernel, in its padded layout,
    needs no more wavefronts than its bytes demand; the plain layout (no
    padding) does not, which checks the model."""
    bad = {}
    for site, width, addrs in seg64_accesses(PM, Q):
        if addrs:
            extra = _wavefronts(addrs, width) - _ideal(addrs, width)
            if extra:
                bad[site] = bad.get(site, 0) + extra
    assert not bad, bad
    plain = [64 * t for t in range(32)]
    assert _wavefronts(plain, 4) > _ideal(plain, 4)
