"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that the
pins in test_oracle_pins.py reject every one of them.

Each mutant is oracle.c with one textual change (a dropped term, a wrong bound, a
flipped comparison, a wrong rounding, a constant typo), compiled into a temporary
directory and swapped in for the duration of the check.  No mutant can read or
write out of bounds: each change keeps every index inside the arrays it touches.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

import oracle
from tests import test_oracle_pins as P
from tests.conftest import read_golden

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "flop drops the row start": ("(int64_t)b_rpt[k + 1] - (int64_t)b_rpt[k]", "(int64_t)b_rpt[k + 1]"),
    "nnz never deduplicates": ("if (mark[c] != stamp) {", "if (mark[c] != stamp + 1) {"),
    "marker stamp is the row id": ("int64_t stamp = r; /* unique for this visit */", "int64_t stamp = i;"),
    "marker stamp never changes": ("int64_t stamp = r; /* unique for this visit */", "int64_t stamp = 0;"),
    "prediction floors": ("return (a + b - 1) / b;", "return a / b;"),
    "reference drops M": ("(u128)(uint64_t)z * (u128)(uint64_t)M;", "(u128)(uint64_t)z;"),
    "reference drops |S|": ("(u128)(uint64_t)F * (u128)(uint64_t)n_ids;", "(u128)(uint64_t)F;"),
    "sample comparison flipped": ("orc_h32(seed, (uint64_t)i) < threshold", "orc_h32(seed, (uint64_t)i) > threshold"),
    "sample comparison inclusive": ("orc_h32(seed, (uint64_t)i) < threshold", "orc_h32(seed, (uint64_t)i) <= threshold"),
    "prediction divides before multiplying": (
        "p = (int64_t)ceil_div_u128((u128)(uint64_t)flop[i] * (u128)(uint64_t)z, (u128)(uint64_t)f);",
        "p = (int64_t)((u128)(uint64_t)flop[i] * ceil_div_u128((u128)(uint64_t)z, (u128)(uint64_t)f));"),
    "prediction swaps z* and f*": (
        "p = (int64_t)ceil_div_u128((u128)(uint64_t)flop[i] * (u128)(uint64_t)z, (u128)(uint64_t)f);",
        "p = (int64_t)ceil_div_u128((u128)(uint64_t)flop[i] * (u128)(uint64_t)f, (u128)(uint64_t)z);"),
    "offsets start at one": ("  offsets[0] = 0;\n  for (int64_t i = 0; i < M; ++i) {\n    int64_t p;\n    if (f == 0)",
                             "  offsets[0] = 1;\n  for (int64_t i = 0; i < M; ++i) {\n    int64_t p;\n    if (f == 0)"),
    "hash constant typo": ("0xbf58476d1ce4e5b9ull", "0xbf58476d1ce4e5b8ull"),
    "draw scales by M/2": ("* (uint64_t)M) >> 32", "* (uint64_t)M) >> 33"),
    "sample_num rounds up": ("int64_t s = (3 * M) / 1000;", "int64_t s = (3 * M + 999) / 1000;"),
    "scan subtracts": ("(u128)(uint64_t)f);\n    pred[i] = p;\n    offsets[i + 1] = offsets[i] + p;",
                       "(u128)(uint64_t)f);\n    pred[i] = p;\n    offsets[i + 1] = offsets[i] - p;"),
    "symbolic offsets stop a row early": ("for (int64_t i = 0; i < M; ++i) offsets[i + 1] = offsets[i] + nnz[i];",
                                          "for (int64_t i = 0; i + 1 < M; ++i) offsets[i + 1] = offsets[i] + nnz[i];"),
    "empty sample not flagged": ("if (f == 0) status |= ORC_WARN_EMPTY_SAMPLE;", ""),
    "numeric overwrites the sum": ("            acc[c] += prod;", "            acc[c] = prod;"),
    "numeric squares A's value": ("const double prod = a * (double)b_val[t];", "const double prod = a * a;"),
    "numeric counts each column once": ("            terms[c] += 1;", "            terms[c] = 1;"),
    "numeric leaves rows unsorted": ("        qsort(list, (size_t)n, sizeof(int32_t), orc_cmp_i32);\n", ""),
    "numeric |.| keeps the sign": ("acc_abs[c] += prod < 0.0 ? -prod : prod;", "acc_abs[c] += prod;"),
    "sampled flop uses first row": ("for (int64_t r = 0; r < n_ids; ++r) f += flop[ids[r]];\n  int64_t status = 0;\n  if (f == 0)",
                                    "for (int64_t r = 0; r < n_ids; ++r) f += flop[ids[0]];\n  int64_t status = 0;\n  if (f == 0)"),
}


def _independent_pins():
    """Pins that tie the oracle to something other than its own formulas: known
    answers, brute force, closed forms, distributions and printed values."""
    g = read_golden
    yield lambda: P.test_splitmix64_known_answers(g)
    yield P.test_bernoulli_threshold_extremes
    yield P.test_bernoulli_membership_matches_hash
    yield P.test_bernoulli_threshold_is_strict
    yield lambda: P.test_paper_sample_num(g)
    yield P.test_paper_draw_mapping_covers_rows_in_order
    yield lambda: P.test_flop_and_nnz_against_dense_product((17, 33, 9), 0.3)
    yield lambda: P.test_laplacian_2d_closed_form(9)
    yield P.test_periodic_laplacian_uniform_rows
    yield lambda: P.test_dense_blocks(7)
    yield P.test_reference_design_uniform_rows
    yield P.test_rounding_up_worked_example
    yield lambda: P.test_numeric_against_dense_product((17, 33, 9), 0.5)
    yield lambda: P.test_numeric_laplacian_squared_closed_form(8)
    yield P.test_numeric_sum_identity
    yield P.test_empty_sample_falls_back_to_flop
    yield P.test_paper_draw_counts_repeats


def _pins():
    """Every pin: the independent ones, then the invariant checks that restate
    the ceiling and the draw formula row by row."""
    yield from _independent_pins()
    yield P.test_paper_draw_rows_in_range
    for name in ("lap64", "er", "rmat", "rect"):
        yield lambda n=name: P.test_prediction_invariants(n, oracle.BERNOULLI)
        yield lambda n=name: P.test_prediction_invariants(n, oracle.PAPER_DRAW)


@pytest.fixture(scope="module")
def tmpdir_mod():
    d = tempfile.mkdtemp(prefix="oracle-mutants-")
    yield d
    shutil.rmtree(d, ignore_errors=True)


def _mutant_library(name, tmpdir):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not unique"
    path_c = os.path.join(tmpdir, f"m{abs(hash(name))}.c")
    path_so = path_c[:-2] + ".so"
    if not os.path.exists(path_so):
        with open(path_c, "w") as f:
            f.write(src.replace(old, new))
        subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", path_c, "-o", path_so], check=True)
    return path_so


def _rejected_by(pins, path_so):
    prev = oracle.use_library(path_so)
    try:
        for pin in pins:
            try:
                pin()
            except AssertionError:
                return True
    finally:
        oracle.restore_library(prev)
    return False


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmpdir_mod):
    assert _rejected_by(_pins(), _mutant_library(name, tmpdir_mod)), f"no pin rejects the mutant {name!r}"


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_independent_pins_alone_reject_mutant(name, tmpdir_mod):
    # Without the checks that restate a formula of the oracle (the ceiling and
    # the draw mapping recomputed row by row), each mutant must still fail a pin
    # tied to something else: a closed form, a distribution, a worked example.
    assert _rejected_by(_independent_pins(), _mutant_library(name, tmpdir_mod)), \
        f"only a restating check rejects the mutant {name!r}"


def test_unmutated_oracle_passes_the_same_pins():
    for pin in _pins():
        pin()
