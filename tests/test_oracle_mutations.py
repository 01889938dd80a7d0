"""Pin strength: each planted mistake in the oracle (ORC_MUT=k, built from the
same C source on the CPU) must make at least one pin fail."""
import pytest

import oracle
import pins

MUTATIONS = {
    1: "merge ties go to the right list (unstable)",
    2: "float32 negatives not bit-inverted",
    3: "last item left out of the scatter bounds",
    4: "rest of the right list dropped in a merge",
    5: "bubble sort inner loop one short",
    6: "odd-even compare-split one round short",
    7: "unpaired last run not carried in the merge tree",
    8: "int32 sign bit not flipped",
}


@pytest.mark.parametrize("k", sorted(MUTATIONS), ids=lambda k: f"mut{k}")
def test_planted_mistake_is_caught(k, tmp_path):
    lib = oracle.load(mutation=k, out_dir=str(tmp_path))
    failed = pins.run_pins(lib, stop_at_first=True)
    assert failed, f"no pin caught planted mistake {k}: {MUTATIONS[k]}"
