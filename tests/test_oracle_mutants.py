"""The pins catch plausible mistakes in the oracle.

Each case copies oracle.c, plants one mistake of the kind a transcription error makes (a dropped
term, a wrong sign, index or exponent, a transposed operand, a skipped stage), compiles the copy
and runs every pin of oracle_pins.py against it in a child process.  The case passes only if at
least one pin fails.  The real oracle is never modified.
"""
import os
import subprocess
import sys
import textwrap

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "butterfly_add_becomes_sub": ("mod_add(&A[k + j], &u, &t, Q);", "mod_sub(&A[k + j], &u, &t, Q);"),
    "butterfly_sub_operands_swapped": ("mod_sub(&A[k + j + half], &u, &t, Q);",
                                       "mod_sub(&A[k + j + half], &t, &u, Q);"),
    "stage_root_wrong_exponent": ("mod_pow_u64(&wm, w, N / m, Q);", "mod_pow_u64(&wm, w, N / half, Q);"),
    "last_stage_dropped": ("for (unsigned s = 1; s <= log2n; ++s)", "for (unsigned s = 1; s < log2n; ++s)"),
    "twist_power_not_advanced": ("                mod_mul(&f, &f, root, Q);\n", "\n"),
    "negacyclic_uses_psi_not_psi2": ("mod_mul(&w, root, root, Q); /* w = psi^2 */", "w = *root;"),
    "inverse_scale_dropped": ("            f = n_inv;\n", "            bn_set_u64(&f, 1);\n"),
    "untwist_uses_psi": ("mod_mul(&f, &f, &psi_inv, Q);", "mod_mul(&f, &f, root, Q);"),
    "bitrev_order_not_applied": ("        if (flags & OR_BITREV) permute_bit_reversed(A, log2n);\n    } else {",
                                 "    } else {"),
    "mul_carry_dropped": ("            carry = t >> 32;\n        }\n        for (int k = i + BN_LIMBS;",
                          "            carry = 0;\n        }\n        for (int k = i + BN_LIMBS;"),
    "sub_borrow_dropped": ("borrow = (d >> 63) & 1;", "borrow = 0;"),
    "mod_compare_strict": ("if (bn_cmp(&rem, q) >= 0) bn_sub(&rem, &rem, q);",
                           "if (bn_cmp(&rem, q) > 0) bn_sub(&rem, &rem, q);"),
    "vsub_operands_transposed": ("case OR_VSUB: mod_sub(&R, &A, &B, &Q); break;",
                                 "case OR_VSUB: mod_sub(&R, &B, &A, &Q); break;"),
    "axpy_scales_y": ("mod_mul(&T, &S, &A, &Q);", "mod_mul(&T, &S, &B, &Q);"),
    "dft_exponent_indices_swapped": ("(uint64_t)(((2 * k + 1) * j) % ord);", "(uint64_t)(((2 * j + 1) * k) % ord);"),
    "point_exponent_missing_one": ("mod_pow_u64(&step, &g, cyclic ? k : 2 * k + 1, &Q);",
                                   "mod_pow_u64(&step, &g, cyclic ? k : 2 * k, &Q);"),
    "negacyclic_fold_sign": ("                mod_sub(&acc, &acc, &p, &Q);", "                mod_add(&acc, &acc, &p, &Q);"),
    "pow_skips_multiply": ("if (bn_bit(e, i)) mod_mul(&acc, &acc, &base, q);", "if (bn_bit(e, i) && i) mod_mul(&acc, &acc, &base, q);"),
    "high_word_lost_on_load": ("bn_set_words(a, p + (size_t)width * i, width);",
                               "bn_set_words(a, p + (size_t)width * i, 1);"),
}

RUNNER = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import oracle
    from tests import oracle_pins
    O = oracle.Oracle({lib!r})
    for pin in oracle_pins.PINS:
        try:
            pin(O)
        except Exception as e:
            print("caught by", pin.__name__, type(e).__name__)
            sys.exit(1)
    sys.exit(0)
""")


def test_every_mutation_applies_once():
    src = open(oracle.SOURCE).read()
    for name, (orig, _) in MUTANTS.items():
        assert src.count(orig) == 1, name


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    orig, mutated = MUTANTS[name]
    src = open(oracle.SOURCE).read()
    assert src.count(orig) == 1
    mpath = tmp_path / "oracle_mutant.c"
    mpath.write_text(src.replace(orig, mutated))
    lib = oracle.build(str(mpath), str(tmp_path / "liboracle_mutant.so"), force=True)
    r = subprocess.run([sys.executable, "-c", RUNNER.format(root=ROOT, lib=lib)], capture_output=True, text=True,
                       timeout=300)
    # a crash (negative return code) also counts as caught; exit 0 means every pin passed
    assert r.returncode != 0, f"mutant {name} survived every pin:\n{r.stdout}\n{r.stderr}"
