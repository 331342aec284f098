"""The oracle's pins must catch plausible mistakes. Each case plants one
mistake in a scratch copy of the oracle's C source (on the CPU: a dropped
term, a wrong sign, index or tag, a flipped comparison), rebuilds the copy
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
     "j = (jo + 1) % c->num_hashes;", "j = (j + 1) % c->num_hashes;"),
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
    env = dict(os.environ, PYTHONPATH=str(dst))
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
