"""Host-side check of the shared-memory addressing of the length-specialised
FFT passes (no GPU).

The passes keep NT transforms of length L = 2^B interleaved in padded shared
memory, element (pos, n) at pad(pos) * NT + n with pad(x) = x + (x >> PS).
Their Stockham stages (radix 2^(B mod 4) first, then radix 16; thread t of a
transform holds 16 values) read positions t + c and write positions bo(t) + c,
c a compile-time constant, and the kernels address both as a per-thread base
plus an immediate: pad(base + c) = pad(base) + pad(c).  This test checks that
identity, and that the stage outputs are the Stockham output positions, for
every length, block width and stage the kernels are compiled for, with the
pad shift rule the kernels use.
"""
import pytest


def pad_shift(L, NT):
    # the rule of kspec::pad_shift (and of the generic radix-16 passes)
    if L >= 4096:
        return 4
    if L == 2048:
        return 4 if NT == 1 else 3
    if NT >= 4:
        return 2
    if NT == 2:
        return 3
    return 4


@pytest.mark.parametrize("B", range(6, 14))
@pytest.mark.parametrize("NT", [1, 2, 4, 8])
def test_padded_offsets_split_into_base_plus_constant(B, NT):
    L = 1 << B
    LT = L // 16
    if NT * LT > 1024:
        pytest.skip("not compiled: more than 1024 threads per block")
    PS = pad_shift(L, NT)
    R0 = (1 << (B % 4)) if B % 4 else 16
    S = (B + 3) // 4

    def pad(x):
        return x + (x >> PS)

    seen_out = set()
    for s in range(S):
        R = R0 if s == 0 else 16
        Ns = 1 if s == 0 else R0 * 16 ** (s - 1)
        assert LT % Ns == 0
        outs = set()
        for t in range(LT):
            k = t & (Ns - 1)
            bo = (t - k) * R + k
            for u in range(16 // R):
                j = t + u * LT
                for r in range(R):
                    c_in = u * LT + r * (L // R)
                    assert pad(t + c_in) == pad(t) + pad(c_in)
                    c_out = u * LT * R + r * Ns
                    # the Stockham output position of butterfly j, input r
                    assert bo + c_out == (j - (j & (Ns - 1))) * R + (j & (Ns - 1)) + r * Ns
                    assert pad(bo + c_out) == pad(bo) + pad(c_out)
                    outs.add(bo + c_out)
        # every stage writes each position exactly once
        assert outs == set(range(L))
        seen_out |= outs
    # the last stage's stride is L/16, so thread t ends with positions t + m L/16
    assert R0 * 16 ** (S - 2) == LT if S > 1 else True
