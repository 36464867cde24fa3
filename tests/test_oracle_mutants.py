"""The oracle's pins catch plausible mistakes.

Every case below plants one mistake in a copy of oracle.c: a dropped term, a
wrong sign, index or operand, a boundary off by one, a tie broken the other
way. The test builds the copy and runs the pin suite (test_oracle_pins.py)
against it with ORACLE_LIBRARY pointing at the copy. The pins must fail on
every mutant. The real oracle is never touched. Each mutant keeps every memory
access in bounds, so a failure is a failed assertion and not a crash, and each
changes what the oracle computes (a planted change that cannot alter any
result, such as narrowing a codec's search range below a value a branch before
it already handles, is not a mutant).
"""
import concurrent.futures
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (what goes wrong, where in the oracle, the correct text, the planted text)
MUTANTS = [
    ("inner product drops the last common dim", "Def. 2",
     "while (a < xn && b < qn) {", "while (a + 1 < xn && b < qn) {"),
    ("inner product ignores the document value's sign", "Def. 2",
     "else { s += xv[a] * qv[b]; a++; b++; }", "else { s += fabs(xv[a]) * qv[b]; a++; b++; }"),
    ("inner product adds instead of multiplying", "Def. 2",
     "else { s += xv[a] * qv[b]; a++; b++; }", "else { s += xv[a] + qv[b]; a++; b++; }"),
    ("equal scores ranked by the higher id", "result order",
     "(a.s == b.s && a.id < b.id)", "(a.s == b.s && a.id > b.id)"),
    ("heap sifts the best hit to the root", "Alg. 2 heap H",
     "if (better(H->h[p], H->h[i])) {", "if (better(H->h[i], H->h[p])) {"),
    ("explicit zeros kept as entries", "Def. 1",
     "if (row[t].v == 0.0) continue;", "if (row[t].v != row[t].v) continue;"),
    ("duplicate dims accepted", "Def. 1",
     "if (row[t].j == row[t - 1].j)", "if (row[t].j < row[t - 1].j)"),
    ("alpha-mass boundary is strict", "alpha-mass subvector",
     "if (prefix >= target) { r = t + 1; break; }", "if (prefix > target) { r = t + 1; break; }"),
    ("alpha-mass keeps one entry too many", "alpha-mass subvector",
     "if (prefix >= target) { r = t + 1; break; }",
     "if (prefix >= target) { r = t + 2 < n ? t + 2 : n; break; }"),
    ("alpha-mass orders entries by signed value", "mass of a vector",
     "for (int64_t t = 0; t < n; t++) { work[t].a = fabs(val[t]); work[t].j = dim[t]; work[t].pos = t; }\n"
     "    qsort(work, (size_t)n, sizeof(orc_mag), cmp_mag);\n    int64_t r;\n",
     "for (int64_t t = 0; t < n; t++) { work[t].a = val[t]; work[t].j = dim[t]; work[t].pos = t; }\n"
     "    qsort(work, (size_t)n, sizeof(orc_mag), cmp_mag);\n    int64_t r;\n"),
    ("alpha-mass breaks equal |x| by the higher dim", "alpha-mass order pi",
     "return (a->j > b->j) - (a->j < b->j);", "return (a->j < b->j) - (a->j > b->j);"),
    ("alpha = 1 left to FP64 prefix sums", "alpha-mass subvector",
     "if (alpha >= 1.0) {", "if (alpha > 1.0) {"),
    ("vector number pruning keeps one entry too many", "Sec. 4.1 VNP",
     "int64_t r = n < vn ? n : vn;", "int64_t r = n < vn + 1 ? n : vn + 1;"),
    ("list pruning keeps one entry too many", "Sec. 4.1 LP",
     "if (t < n_keep) lkeep[lw[t].pos] = 1;", "if (t <= n_keep) lkeep[lw[t].pos] = 1;"),
    ("list pruning breaks equal |x| by the higher doc", "Sec. 4.1 LP",
     "return (a->doc < b->doc) ? -1 : (a->doc > b->doc);", "return (a->doc > b->doc) ? -1 : (a->doc < b->doc);"),
    ("list pruning ranks signed values", "Sec. 4.1 LP",
     "lw[t].a = fabs(xval[b + t]);", "lw[t].a = xval[b + t];"),
    ("mass-list pruning skips the alpha-mass step", "Sec. 5 ablation",
     "(prune == ORC_PRUNE_MASS || prune == ORC_PRUNE_MASS_LIST) ? alpha : 1.0;",
     "(prune == ORC_PRUNE_MASS) ? alpha : 1.0;"),
    ("window slot off by one", "Alg. 2",
     "int64_t m = I->pid[p] % lambda;", "int64_t m = (I->pid[p] + 1) % lambda;"),
    ("accumulation overwrites the slot", "Alg. 2",
     "A[m] = A[m] + prod;", "A[m] = prod;"),
    ("product drops the query weight", "Alg. 2",
     "double prod = q * I->pval[p];", "double prod = I->pval[p];"),
    ("last window never scanned", "Alg. 2",
     "for (int64_t w = 0; w < sigma; w++) {", "for (int64_t w = 0; w + 1 < sigma; w++) {"),
    ("score window not reset between windows", "Alg. 2",
     "}\n            A[m] = 0.0;\n", "}\n"),
    ("reorder keeps the coarse scores", "Alg. 4",
     "orc_hit x = { orc_inner_product(I->D, i, Q, r), i };", "orc_hit x = { hs[t], i };"),
    ("reorder scores with the pruned query", "Alg. 4",
     "orc_hit x = { orc_inner_product(I->D, i, Q, r), i };",
     "orc_hit x = { inner_product(I->D->dim + I->D->ptr[i], I->D->val + I->D->ptr[i], "
     "I->D->ptr[i + 1] - I->D->ptr[i], pd, pv, pn), i };"),
    ("reorder draws only k candidates", "Alg. 4",
     "int64_t nh = precise_search(I, pd, pv, pn, gamma, hid, hs);",
     "int64_t nh = precise_search(I, pd, pv, pn, k < gamma ? k : gamma, hid, hs);"),
    ("beta ignored", "Alg. 4",
     "int64_t rq = alpha_mass(qd, qv, qn, beta, kpos, work);",
     "int64_t rq = alpha_mass(qd, qv, qn, 1.0, kpos, work);"),
    ("round-to-nearest ties go up", "IEEE 754 / OCP rounding",
     "return (code_lo & 1) ? code_lo + 1 : code_lo;", "return code_lo + 1;"),
    ("binary16 overflows to inf one step late", "IEEE 754 binary16",
     "if (a >= 65520.0) return sign | 0x7C00;", "if (a > 65520.0) return sign | 0x7C00;"),
    ("binary16 subnormals scaled by 2^-25", "IEEE 754 binary16",
     "if (e == 0) v = ldexp((double)m, -24);", "if (e == 0) v = ldexp((double)m, -25);"),
    ("E4M3 exponent bias 8", "OCP E4M3",
     "else v = ldexp((double)(8 + m), e - 10);", "else v = ldexp((double)(8 + m), e - 11);"),
    ("E4M3 overflow gives NaN", "OCP E4M3",
     "if (a >= 448.0) return (uint8_t)(sign | 0x7E);", "if (a >= 448.0) return (uint8_t)(sign | 0x7F);"),
    ("E4M3 list scale over 240", "per-list FP8 scale",
     "volatile float sc = amax / 448.0f;", "volatile float sc = amax / 240.0f;"),
    ("binary16 posting values stored unrounded", "reduced-precision lists",
     "for (int64_t t = 0; t < P; t++) I->pval[t] = (double)orc_f16_decode(orc_f16_encode((float)I->pval[t]));",
     ""),
    ("dim == d accepted", "Def. 1",
     "if (j < 0 || j >= d || !isfinite(v))", "if (j < 0 || j > d || !isfinite(v))"),
    ("non-finite values accepted", "Def. 1",
     "if (j < 0 || j >= d || !isfinite(v))", "if (j < 0 || j >= d)"),
    ("brute force skips the last document", "Def. 3",
     "    for (int64_t i = 0; i < D->n; i++) {\n        orc_hit x = { orc_inner_product(D, i, Q, r), i };",
     "    for (int64_t i = 0; i + 1 < D->n; i++) {\n        orc_hit x = { orc_inner_product(D, i, Q, r), i };"),
    ("inner product advances the wrong cursor", "Def. 2",
     "if (xd[a] < qd[b]) a++;\n        else if (xd[a] > qd[b]) b++;",
     "if (xd[a] < qd[b]) b++;\n        else if (xd[a] > qd[b]) a++;"),
    ("results drained worst first", "result order",
     "if (better(a, b)) return -1;\n    if (better(b, a)) return 1;",
     "if (better(a, b)) return 1;\n    if (better(b, a)) return -1;"),
    ("list offsets miss the last prefix step", "Alg. 1",
     "for (int64_t s = 0; s < d * sigma; s++) I->seg[s + 1] += I->seg[s];",
     "for (int64_t s = 0; s + 1 < d * sigma; s++) I->seg[s + 1] += I->seg[s];"),
    ("list pruning leaves the kept counts unchanged", "Sec. 4.1 LP",
     "else I->kept_count[lw[t].doc]--;", ""),
    ("E4M3 subnormals scaled by 2^-10", "OCP E4M3",
     "if (e == 0) v = ldexp((double)m, -9);", "if (e == 0) v = ldexp((double)m, -10);"),
]


def _run_mutant(tmp_path, n, mutant):
    name, _, old, new = mutant
    with open(oracle._SRC, encoding="utf-8") as f:
        src = f.read()
    if src.count(old) != 1:
        return name, f"site found {src.count(old)} times"
    d = tmp_path / f"m{n:02d}"
    d.mkdir()
    c, so = str(d / "oracle.c"), str(d / "liboracle.so")
    with open(c, "w", encoding="utf-8") as f:
        f.write(src.replace(old, new))
    oracle.compile_library(c, so)
    env = dict(os.environ, ORACLE_LIBRARY=so, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    if r.returncode == 1:
        return name, None                               # a pin failed: caught
    if r.returncode == 0:
        return name, "every pin passed"
    return name, f"pytest exit {r.returncode}: {r.stdout[-300:]}"


def test_every_planted_mistake_fails_a_pin(tmp_path):
    assert len({m[0] for m in MUTANTS}) == len(MUTANTS)
    oracle.build()
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda a: _run_mutant(tmp_path, *a), enumerate(MUTANTS)))
    missed = [f"{name}: {why}" for name, why in results if why is not None]
    assert not missed, "mutants the pins did not catch:\n" + "\n".join(missed)


def test_the_unmutated_copy_passes(tmp_path):
    """The same harness on an unchanged copy passes: failures above come from the planted mistakes."""
    name, why = _run_mutant(tmp_path, 99, ("unchanged", "", "#include <math.h>", "#include <math.h>"))
    assert why == "every pin passed"
