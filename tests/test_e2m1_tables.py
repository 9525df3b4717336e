"""The e2m1 codes of integer genotypes and slice digits (csrc/mixed.cu) against the e2m1 format's
definition: bit 3 the sign, bits 2-1 the exponent e, bit 0 the mantissa m; value m/2 when e = 0,
else (1 + m/2) 2^(e-1).  The table codes the integers -8..7 and the mask marks those with no code;
slice digits in [-4, 4] use the closed form |d| + min(|d|, 2)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def e2m1_value(code):
    s, e, m = (code >> 3) & 1, (code >> 1) & 3, code & 1
    v = m / 2 if e == 0 else (1 + m / 2) * 2.0 ** (e - 1)
    return -v if s else v


def constants():
    src = open(os.path.join(ROOT, "paper_1210_7683_gb300", "csrc", "mixed.cu")).read()
    codes = int(re.search(r"kE2m1Codes = 0x([0-9A-Fa-f]+)ull", src).group(1), 16)
    bad = int(re.search(r"kE2m1Bad = 0x([0-9A-Fa-f]+)u", src).group(1), 16)
    return codes, bad


def test_format_has_exactly_these_integers():
    ints = sorted({e2m1_value(c) for c in range(16) if e2m1_value(c) == int(e2m1_value(c))})
    assert ints == [-6, -4, -3, -2, -1, 0, 1, 2, 3, 4, 6]


def test_genotype_table_and_mask():
    codes, bad = constants()
    representable = {int(e2m1_value(c)) for c in range(16) if e2m1_value(c) == int(e2m1_value(c))}
    for x in range(-8, 8):
        u = x + 8
        if x in representable:
            assert not (bad >> u) & 1, x
            assert e2m1_value((codes >> (4 * u)) & 15) == x, x
        else:
            assert (bad >> u) & 1, x


def test_digit_codes_closed_form():
    for d in range(-4, 5):
        a = abs(d)
        code = (a + min(a, 2)) | (8 if d < 0 else 0)
        assert e2m1_value(code) == d


def test_slice_digits_split_into_three_e2m1_digits():
    # q = 64 d0 + 8 d1 + d2 by rounded quotients: every q in [-288, 287], which holds the slices'
    # digits (|q| <= 256), splits into digits in [-4, 4], each exact in e2m1; -289 and 288 do not
    for q in (-289, 288):
        d0 = (q + 32) >> 6
        assert not -4 <= d0 <= 4 or not -4 <= (q - 64 * d0 + 4) >> 3 <= 4
    for q in range(-288, 288):
        d0 = (q + 32) >> 6
        r = q - 64 * d0
        d1 = (r + 4) >> 3
        d2 = r - 8 * d1
        assert 64 * d0 + 8 * d1 + d2 == q
        assert all(-4 <= d <= 4 for d in (d0, d1, d2)), q
