"""Host side of the fused-kernel timeline (no GPU): the per-phase summary and
the occupancy bins of hand-made trace records."""
import numpy as np

from paper_2210_14771_gb300 import timeline
from paper_2210_14771_gb300.api import TRACE_DTYPE


def _records(rows):
    tr = np.zeros(len(rows), dtype=TRACE_DTYPE)
    for i, (g, r, e, ph, cta) in enumerate(rows):
        tr[i] = (g, r, e, ph, 0, cta)
    return tr


def test_summary_of_a_known_timeline():
    # two strips (0-10 us, 0-5 us), a fit tile taken at 5 us released at 10 us
    # ending at 30 us, a mask band taken at 10 us released at 30 us ending at 34 us
    base = 1_000_000
    us = 1000
    tr = _records([(base, base, base + 10 * us, 0, 0),
                   (base, base, base + 5 * us, 0, 1),
                   (base + 5 * us, base + 10 * us, base + 30 * us, 1, 1),
                   (base + 10 * us, base + 30 * us, base + 34 * us, 2, 0)])
    s = timeline.summarise(tr)
    assert s["span_us"] == 34.0 and s["items"] == 4 and s["ctas"] == 2
    assert s["strips"]["n"] == 2 and s["strips"]["last_us"] == 10.0
    assert s["strips"]["wait_us"] == 0.0 and s["strips"]["work_us"] == 7.5
    assert s["fit"]["first_us"] == 5.0 and s["fit"]["wait_us"] == 5.0 and s["fit"]["work_us"] == 20.0
    assert s["mask"]["wait_us"] == 20.0 and s["mask"]["work_us"] == 4.0
    assert s["strips"]["cta_us"] == 15.0
    occ = timeline.occupancy(tr, bin_us=5.0)
    # strips: both in [0, 5), one in [5, 10); fit covers [5, 30); mask [10, 34)
    assert occ["strips"][:3].tolist() == [2.0, 1.0, 0.0]
    assert np.allclose(occ["fit"][:7], [0, 1, 1, 1, 1, 1, 0])
    assert np.allclose(occ["mask"][:7], [0, 0, 1, 1, 1, 1, 0.8])
    # item-time conservation: the bins add up to the items' durations
    for k, name in enumerate(timeline.PHASES):
        m = tr["phase"] == k
        assert np.isclose(occ[name].sum() * 5.0,
                          ((tr["t_end"][m] - tr["t_grab"][m]) / 1e3).sum())
