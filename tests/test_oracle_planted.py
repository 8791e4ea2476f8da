"""The oracle's pins catch plausible mistakes.

Each case copies f2_oracle.c, plants one mistake (a dropped term, a wrong
index, a missing swap), compiles the copy on the CPU and checks that the
pins of tests/test_oracle_pins.py reject it.  The committed oracle is never
modified.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import f2gen
import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "f2_oracle.c")

MUTATIONS = {
    "search-skips-current-row": (
        "for (int64_t i = t; i < n; ++i) {\n            if (getbit(W + i * mu, j)) { piv = i; break; }",
        "for (int64_t i = t + 1; i < n; ++i) {\n            if (getbit(W + i * mu, j)) { piv = i; break; }"),
    "xor-drops-pivot-word": (
        "for (int64_t w = q; w < mu; ++w) row[w] ^= prow[w];",
        "for (int64_t w = q + 1; w < mu; ++w) row[w] ^= prow[w];"),
    "multiplier-not-recorded": (
        "                setbit(Lw + i * lw, t);\n", "\n"),
    "perm-not-swapped": (
        "int32_t tmp = pr[piv]; pr[piv] = pr[t]; pr[t] = tmp;", ""),
    "L-rows-not-swapped": (
        "swap_words(Lw + piv * lw, Lw + t * lw, lw);", ""),
    "pivot-search-drops-rank-one-term": (
        "if (popcount_odd(rk & zc[t])) zc[t] ^= ct | kbit;", "if (popcount_odd(rk & zc[t])) zc[t] ^= kbit;"),
    "pivot-search-condition-drops-reduction": (
        "if (alpha ^ popcount_odd(a[i] & low & ct)) {", "if (alpha) {"),
    "pivot-search-transposed-swap": (
        "const int64_t r1 = R + s, r2 = R + P[k];", "const int64_t r1 = R + s, r2 = R + P[k] + (P[k] > s);"),
    "mmm-transposed-operand": (
        "if (!getbit(A + i * lda, t)) continue;", "if (!getbit(A + t * lda, i)) continue;"),
}


def build_mutant(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", str(path), "-o", str(so)], check=True)
    return oracle.load_library(str(so))


def run_pins():
    """A compact subset of the pins; returns True iff all of them pass."""
    try:
        for code in range(0, 1 << 9, 3):
            bits = np.array([(code >> k) & 1 for k in range(9)], dtype=np.int64).reshape(3, 3)
            out = oracle.ple(f2gen.pack_bits(bits), 3)
            assert out["rank"] == pins.brute_rank(bits)
            pins.check_ple_invariants(bits, out)
        for name, A, m in list(pins.matrices())[:6]:
            bits = pins.bits_of(A, m)
            out = oracle.ple(A, m)
            pins.check_ple_invariants(bits, out)
            for b in (3, 8, 64):
                blk = oracle.blockdecomp(A, m, b)
                assert np.array_equal(blk["perm"], out["perm"])
                assert np.array_equal(blk["pivcols"], out["pivcols"])
                pins.check_figure1_storage(bits, blk, b)
        A = f2gen.uniform(40, 70, 3)
        B = f2gen.uniform(70, 50, 4)
        C = oracle.mmm(A, B, 70, 50)
        assert np.array_equal(pins.bits_of(C, 50), (pins.bits_of(A, 70) @ pins.bits_of(B, 50)) % 2)
    except AssertionError:
        return False
    return True


def test_unmodified_oracle_passes_subset():
    assert run_pins()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, monkeypatch, name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    monkeypatch.setattr(oracle, "_lib", build_mutant(tmp_path, name))
    assert not run_pins(), f"planted mistake '{name}' passed the pins"
