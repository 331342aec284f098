"""The oracle's pins must catch plausible mistakes. Each case plants one
mistake in a scratch copy of the oracle's C source (on the CPU: a dropped
term, a wrong sign, index or tag, a flipped comparison, in the algorithms
and in the invariant checkers), rebuilds the copy
and runs the oracle pin tests against it in a subprocess; at least one pin
must fail. An unmutated copy must pass, so a failure means the mistake, not
the harness."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("Definition 1: ties between levels go to the wrong one",
     "return y1 <= y2; /* x1 == 2, x2 == 1 */", "return y1 < y2; /* x1 == 2, x2 == 1 */"),
    ("secondary entry tag swapped",
     "return (body << 2) | (uint64_t)x;", "return (body << 2) | (uint64_t)(3 - x);"),
    ("inverse permutation drops the round function",
     "uint64_t L = (p >> R) ^ orc_round(c, level, j, r);", "uint64_t L = (p >> R);"),
    ("evicted key continues under the wrong hash",
     "k = orc_cuckoo_decode(c, a, old, &jo);\n        j = (jo + 1) % c->num_hashes;",
     "k = orc_cuckoo_decode(c, a, old, &jo);\n        j = (j + 1) % c->num_hashes;"),
    ("Algorithm 5 ignores the slot order",
     "if (bx < 0 || orc_prec(x, y, bx, by)) {", "if (bx < 0) {"),
    ("round function shifted by one bit",
     "return (A * r + B) >> (64 - n);", "return (A * r + B) >> (63 - n);"),
    ("lookup early stop inverted",
     "if (orc_bucket_has_empty(c, 0, table, a))", "if (!orc_bucket_has_empty(c, 0, table, a))"),
    ("slot index forgets the primary level's slots",
     "c->nb[0] * (uint64_t)B0 + a * (uint64_t)B1 + (uint64_t)y", "a * (uint64_t)B1 + (uint64_t)y"),
    ("cuckoo entry tag off by one",
     "return (body << 2) | (uint64_t)(j + 1);", "return (body << 2) | (uint64_t)j;"),
    ("primary occupancy bit dropped",
     "return (body << 1) | 1ULL;", "return body << 1;"),
    ("enumeration decodes secondary entries with the other hash",
     "return c->compact ? orc_key_from(c, 1, x - 1, a, e >> 2) : e >> 2;",
     "return c->compact ? orc_key_from(c, 1, 2 - x, a, e >> 2) : e >> 2;"),
    ("enumeration decodes primary entries without the flag shift",
     "return c->compact ? orc_key_from(c, 0, 0, a, e >> 1) : e >> 1;",
     "return c->compact ? orc_key_from(c, 0, 0, a, e >> 2) : e >> 1;"),
    # mistakes in the invariant checkers themselves
    ("prefix checker counts every late slot, not every bucket",
     "else if (seen_empty) {\n                bad++;\n                break;",
     "else if (seen_empty) {\n                bad++;"),
    ("order-property checker with the slot order reversed",
     "if (!orc_prec(x2, y2, x, y))", "if (!orc_prec(x, y, x2, y2))"),
    ("order-property checker never visits the secondary level",
     "for (int level = 0; level < 2; level++) {", "for (int level = 0; level < 1; level++) {"),
    ("order-property checker misses a preceding copy of the same key",
     "if (e2 == 0 || e2 == ke[x2]) {", "if (e2 == 0) {"),
    ("order-property checker looks in the wrong bucket",
     "kb[x2] = orc_iceberg_bucket(c, x2, k);", "kb[x2] = orc_iceberg_bucket(c, x, k);"),
    ("chain checker also inspects the entry's own bucket",
     "for (int jj = 0; jj < j; jj++)", "for (int jj = 0; jj <= j; jj++)"),
    ("chain checker skips the first bucket of the chain",
     "for (int jj = 0; jj < j; jj++)", "for (int jj = 1; jj < j; jj++)"),
    ("entries checker accepts a hash index equal to H",
     "ok = x >= 0 && x < c->num_hashes &&", "ok = x >= 0 && x <= c->num_hashes &&"),
    ("entries checker skips the cuckoo address test",
     "orc_address(c, 0, x, k) == a &&", ""),
    ("entries checker skips the secondary address test",
     "orc_iceberg_bucket(c, x, k) == a &&", ""),
    # mistakes in the host-threaded model of the packed-word claim
    ("threaded claim writes the word without a compare-and-swap",
     "        if (__atomic_compare_exchange_n(wp, &old, desired, 0, __ATOMIC_RELAXED,\n"
     "                                        __ATOMIC_RELAXED))\n            return 1;\n"
     "        (*fails)++;",
     "        __atomic_store_n(wp, desired, __ATOMIC_RELAXED);\n        return 1;\n"
     "        (*fails)++;"),
    ("threaded put continues the evicted key under the wrong hash",
     "k = orc_cuckoo_decode(c, a, prev, &jo);\n        j = (jo + 1) % c->num_hashes;",
     "k = orc_cuckoo_decode(c, a, prev, &jo);\n        j = (j + 1) % c->num_hashes;"),
    ("threaded level-2 choice gives ties to the first bucket",
     "int pick1 = y1 < y2;", "int pick1 = y1 <= y2;"),
    ("threaded claim takes a lost field as its own",
     "        if (fld != 0) {\n            *seen = fld;", "        if (fld != 0) {\n            *seen = e;"),
    # mistakes in the level-3 stash
    ("stash put only tries the home position",
     "    for (uint64_t i = 0; i < c->stash; i++) {\n        uint64_t p = (h + i) & (c->stash - 1);\n"
     "        if (st[p] == k)\n            return ORC_FOUND;",
     "    for (uint64_t i = 0; i < 1; i++) {\n        uint64_t p = (h + i) & (c->stash - 1);\n"
     "        if (st[p] == k)\n            return ORC_FOUND;"),
    ("lookup never reaches the stash",
     "if (!hit && !room && c->stash)", "if (!hit && !room && 0)"),
    ("enumeration forgets the stash",
     "if (c->kind == 1 && c->stash) {", "if (c->kind == 1 && 0) {"),
    ("stash home from the wrong constant",
     "orc_mix64(k ^ orc_splitmix(c->seed, 16))", "orc_mix64(k ^ orc_splitmix(c->seed, 15))"),
    ("threaded stash claim without a compare-and-swap",
     "            if (__atomic_compare_exchange_n(sp, &expected, k, 0, __ATOMIC_RELAXED,\n"
     "                                            __ATOMIC_RELAXED))\n                return ORC_PUT;",
     "            __atomic_store_n(sp, k, __ATOMIC_RELAXED);\n                return ORC_PUT;"),
    ("stash checker ignores gaps on the probe path",
     "if (st[q] == 0 || st[q] == k)", "if (st[q] == k)"),
    ("duplicates checker skips the first pair",
     "for (uint64_t i = 1; i < n; i++)\n        if (keys[i] == keys[i - 1])",
     "for (uint64_t i = 2; i < n; i++)\n        if (keys[i] == keys[i - 1])"),
]


def _scratch(tmp_path, old=None, new=None):
    dst = tmp_path / "copy"
    shutil.copytree(os.path.join(ROOT, "oracle"), dst / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    (dst / "tests").mkdir()
    for f in os.listdir(os.path.join(ROOT, "tests")):
        if f == "conftest.py" or (f.startswith("test_oracle_") and f.endswith(".py")
                                  and f != os.path.basename(__file__)):
            shutil.copy(os.path.join(ROOT, "tests", f), dst / "tests" / f)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), dst / "tests" / "golden")
    if old is not None:
        src = dst / "oracle" / "oracle.c"
        text = src.read_text()
        assert text.count(old) == 1, f"mutation anchor not unique: {old!r}"
        src.write_text(text.replace(old, new))
    return dst


def _run_pins(dst) -> int:
    # the scratch oracle first; the package (input generators) from the repo
    env = dict(os.environ, PYTHONPATH=f"{dst}{os.pathsep}{ROOT}")
    r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-q", "-x",
                        "-p", "no:cacheprovider"], cwd=dst, env=env,
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, timeout=600)
    return r.returncode


def test_unmutated_copy_passes(tmp_path):
    assert _run_pins(_scratch(tmp_path)) == 0


@pytest.mark.slow
@pytest.mark.parametrize("what,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(tmp_path, what, old, new):
    assert _run_pins(_scratch(tmp_path, old, new)) != 0, f"no pin caught: {what}"
