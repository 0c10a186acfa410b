"""The compile-time stages' index folding (fft_static.cuh), checked on the CPU for every length,
stage, thread, butterfly and padding period: the shared-memory addresses a stage computes as a
per-thread base plus a compile-time offset equal the padded addresses of the plain Stockham
indices, inputs e = j + q L/R and outputs o = (j / Ns) R Ns + (j mod Ns) + p Ns of butterfly
j = lt + b tpt, and each stage's outputs cover the line exactly once.
"""
import numpy as np
import pytest

# (ED, elements per thread): L = 2^(ED - 1000) in radix-16 stages, L = 3 2^(ED - 2000) in radix-8
# stages and a last radix-3 stage
FAMILIES = [(ed, 16) for ed in range(1008, 1015)] + [(ed, 24) for ed in range(2007, 2013)]


def stages(ed):
    x3 = ed >= 2000
    l2 = ed - 2000 if x3 else ed - 1000
    L = (3 << l2) if x3 else (1 << l2)
    lr = 3 if x3 else 4
    nmain, rem = l2 // lr, l2 % lr
    nst = nmain + (1 if rem else 0) + (1 if x3 else 0)
    out, lns = [], 0
    for s in range(nst):
        R = (1 << lr) if s < nmain else ((1 << rem) if (s == nmain and rem) else 3)
        out.append((R, lns))
        lns += lr if s < nmain else rem
    return L, out


def pidx(e, ps):
    return e + (e >> ps)


@pytest.mark.parametrize("ed,E", FAMILIES)
@pytest.mark.parametrize("ps", [4, 3])  # FP32 (16 x 8 B) and FP64 (8 x 16 B) padding periods
def test_folded_indices_match_the_stockham_indices(ed, E, ps):
    L, st = stages(ed)
    TPT = L // E
    PAD = 1 << ps
    if TPT % PAD:
        pytest.skip("the compile-time lengths need tpt to be a multiple of the padding period")
    lt = np.arange(TPT, dtype=np.int64)
    for R, lns in st:
        Ns, RN = 1 << lns, R << lns
        NB, NBF = E // R, (E // R) * TPT
        assert E % R == 0 and NBF * R == L
        pl = lt + (lt >> ps)
        if Ns <= TPT:
            k0, jq0 = lt & (Ns - 1), lt >> lns
        else:
            k0, jq0 = lt.copy(), np.zeros_like(lt)
        if RN <= PAD:
            x = jq0 * RN
            T0 = x + (x >> ps) + k0
        elif Ns < PAD:
            T0 = jq0 * (RN + RN // PAD) + k0
        else:
            T0 = jq0 * (RN + RN // PAD) + k0 + (k0 >> ps)
        O0 = jq0 * RN + k0
        outs = []
        for b in range(NB):
            j = lt + b * TPT
            for q in range(R):
                c = b * TPT + q * NBF
                assert np.array_equal(pl + c + (c >> ps), pidx(j + q * NBF, ps))
            cb = b * TPT
            ck, cj = cb & (Ns - 1), cb >> lns
            if RN <= PAD:
                Cb = cj * RN + ((cj * RN) >> ps)
            else:
                Cb = cj * (RN + RN // PAD) + ck + (ck >> ps)
            for p in range(R):
                if RN <= PAD:
                    Cp = p * Ns
                elif Ns < PAD:
                    Cp = p * Ns + ((p * Ns) >> ps)
                else:
                    Cp = p * (Ns + Ns // PAD)
                o = O0 + cj * RN + ck + p * Ns
                direct = (j // Ns) * RN + (j % Ns) + p * Ns
                assert np.array_equal(o, direct)
                assert np.array_equal(T0 + Cb + Cp, pidx(direct, ps))
                outs.append(direct)
        allo = np.sort(np.concatenate(outs))
        assert np.array_equal(allo, np.arange(L))
