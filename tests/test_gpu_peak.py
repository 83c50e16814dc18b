"""The FP64 FMA rate probe (ssg_measure_fp64_rate), the denominator of the
FP64-bound rooflines: it measures a rate that scales with the work (twice
the iterations take twice the time, so launch overhead is negligible) and
refuses bad arguments."""

import pytest

pytestmark = pytest.mark.gpu


def test_fp64_rate_probe():
    from paper_2108_13162_gb300 import build as ssg_build
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Context

    ssg_build.build()
    ctx = Context(0)
    t1, ms1 = ssg.ssg_measure_fp64_rate(ctx.h, 4000, 3)
    t2, ms2 = ssg.ssg_measure_fp64_rate(ctx.h, 8000, 3)
    assert t1 > 0 and t2 > 0
    assert 1.7 <= ms2 / ms1 <= 2.3, (ms1, ms2)
    assert abs(t2 / t1 - 1.0) <= 0.15, (t1, t2)
    with pytest.raises(ssg.SSGError):
        ssg.ssg_measure_fp64_rate(ctx.h, 0, 3)
    ctx.close()
