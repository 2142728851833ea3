"""The 2-D variant's host-only band schedule (csc2d_plan, include/csc2d.h)
equals the 2-D oracle's band cut and phase count (rows cut into bands, the
paper's conclusion; segments and phases of Sec. 2.2 taken along rows)."""
import pytest

from oracle import csc2d
from paper_1705_10087_gb300 import build, capi


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load()


@pytest.mark.parametrize("Hz,h,M", [(121, 8, 8), (121, 8, 4), (121, 8, 16), (36, 5, 6), (36, 5, 1),
                                    (249, 8, 17), (7, 1, 7), (1000, 16, 33)])
def test_band_plan_matches_oracle(lib, Hz, h, M):
    Mo, c, starts = capi.csc2d_plan(Hz, h, M)
    assert Mo == M
    assert c == csc2d.phase_count(Hz, M, h)
    assert list(starts) == [csc2d.band_start(Hz, M, m) for m in range(M + 1)]


def test_band_plan_automatic_and_rejects(lib):
    M, c, starts = capi.csc2d_plan(249, 8, 0)
    assert min(b - a for a, b in zip(starts[:-1], starts[1:])) >= 2 * 8 - 2 and c == 2
    with pytest.raises(capi.CscError):
        capi.csc2d_plan(10, 4, 11)
