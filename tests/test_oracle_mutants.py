"""The pins catch plausible mistakes in the oracle: each ORACLE_MUTANT build
(oracle/oracle.cpp) plants one -- a wrong operator, a dropped product-rule
term, a transposed head, a missing clamp, a wrong tie-break or update policy,
a skipped filter or join check, early stopping, samples that join -- and the
pin suite must fail against every one of them (and pass against the oracle)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MUTANTS = {
    1: "max-min (x) takes the larger tag",
    2: "add-mult (+) without the clamp to 1",
    3: "diff-max-min ties go to the larger input-fact id",
    4: "diff-add-mult product rule drops its second term",
    5: "diff-add-mult derivative survives a clamped (+)",
    6: "rule filters ignored",
    7: "a variable bound earlier in the body is not compared",
    8: "iteration stops after the second round",
    9: "max-min keeps the first tag of a key",
    10: "sample ids ignored (samples join)",
    11: "first two head columns transposed",
    12: "diff-max-min (x) keeps the greater operand",
    13: "top-1-proofs union keeps a shared fact twice",
    14: "top-1-proofs (+) keeps the less likely proof",
    15: "'<' admits equality",
    16: "subtraction with its operands swapped",
    17: "strata run in reverse dependency order",
    18: "mutually recursive relations split into separate strata",
    19: "one loop over every rule, strata ignored",
}


def run_pins(mutant: int) -> subprocess.CompletedProcess:
    env = dict(os.environ, ORACLE_MUTANT=str(mutant))
    return subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q", "-p", "no:cacheprovider"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_fail_on_mutant(mutant):
    r = run_pins(mutant)
    # exit code 1 = some test failed (not an error in collection or usage)
    assert r.returncode == 1, (MUTANTS[mutant], r.returncode, r.stdout[-2000:])
