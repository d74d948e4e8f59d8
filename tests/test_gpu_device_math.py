"""Device helpers with a definition of their own, checked directly on the GPU: the logarithm of the
Sinkhorn column updates (log2 b_k - log2 cs_k = -log2(cs_k / b_k), an argument near 1 in a
converging solve), evaluated for every float of its short path."""
import pytest

from gpu_util import require_gpu
from paper_2406_10262_gb300 import fairrank as fr

pytestmark = pytest.mark.gpu


def test_log2_near_one_matches_log2_over_every_float_of_its_range():
    """For |y - 1| < 2^-5 the helper sums the Taylor series of ln(1 + t) / ln 2 through t^6
    (truncation below 2^-30 relative) in FP32 Horner form. Against log2 in double precision its
    relative error must stay within a few FP32 units in the last place (2^-22) -- the same order as
    log2f's own -- and log2(1) must be exactly 0."""
    require_gpu()
    r = fr.check_log2_near1()
    assert r["nonzero_at_one"] == 0
    assert r["max_rel_err"] <= 2.0 ** -22, r
    assert r["max_rel_err"] <= 4.0 * max(r["log2f_max_rel_err"], 2.0 ** -24), r
