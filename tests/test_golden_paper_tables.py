"""Golden values printed in the paper (tests/golden/ngc7683_fit_tables.json, cited there):
the NGC 7683 fit tables of Sec. 3.1 and App. C.  They pin two inputs of this library to the
paper: the prior ranges synth.prior_box uses for the paper's own slots, and the paper-like
parameter vector synth.NGC7683_LIKE (the SPS fit's posterior medians), from which
fit.truth_two_discs builds the synthetic galaxy of the model-selection run."""
import json
import math
import os

import pytest

from paper_2205_06819_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "golden", "ngc7683_fit_tables.json")) as f:
        return json.load(f)


def test_prior_box_uses_the_papers_ranges_for_its_own_slots(golden):
    pr = golden["prior_ranges"]
    box = synth.prior_box(2, halo_kind=1)
    deg = math.pi / 180
    assert tuple(box[2]) == pytest.approx((pr["PA"][0] * deg, pr["PA"][1] * deg))
    assert tuple(box[9]) == tuple(pr["k1"]) and tuple(box[17]) == tuple(pr["k2"])
    assert tuple(box[10]) == tuple(pr["MLb"]) and tuple(box[11]) == tuple(pr["MLd1"])
    assert tuple(box[18]) == tuple(pr["MLd2"])
    assert tuple(box[12]) == tuple(pr["logMh"]) and tuple(box[13]) == tuple(pr["logRh"])


def test_paper_like_vector_is_the_sps_fit(golden):
    t = golden["sps_fit"]
    v = synth.NGC7683_LIKE
    assert v[2] == pytest.approx(t["PA"] * math.pi / 180)
    assert math.sin(v[3]) == pytest.approx(t["sin_i"])
    assert (v[4], v[5], v[7], v[8], v[15], v[16]) == (t["logMb"], t["logRb"], t["logMd1"], t["logRd1"],
                                                      t["logMd2"], t["logRd2"])
    assert (v[10], v[11], v[18], v[9], v[17]) == (t["MLb"], t["MLd1"], t["MLd2"], t["k1"], t["k2"])
