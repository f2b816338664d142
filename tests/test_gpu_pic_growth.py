"""Measured NCI growth of drifting-plasma PIC runs (the library's PIC step on the
Table 1 setup: 256 x 256 cells of 0.2, periodic, gamma = 50, n/n_p = 100, 8 + 8
particles per cell, quadratic shapes) against the root solver's prediction over
the run's own modes, and the Sec. 4 strategies: a low-pass filter of the current
removes the fast (0, +-1) modes; a smaller time step lowers the (0, 0) growth; the
printed k1 modification removes the (0, 0) modes (Fig. 3b: the E2 energy stays at
the noise level until the slower (+-1, +-2) modes grow, and with cubic shapes
those do not grow either).  Measured growth = the fastest clean exponential of the
E2 energy (pic.growth_rate); the prediction includes every alias the run can show
(mu = -1..1, nu1 = -2..2)."""
import numpy as np
import pytest

from gpu_util import hyb_module, need_gpu

pytestmark = pytest.mark.gpu

# measured / predicted bounds: the Appendix takes the charge-conserving current in the
# dt -> 0 limit; measured rates agree to 1 % at dt = 0.04 and come out 15-35 % above
# the prediction at dt = 0.08
HI, LO = 1.5, 0.6


def _case(w, steps, kmod=None):
    from paper_1502_01376_gb300 import pic
    h = pic.run(w, steps=steps, every=10, kmod=kmod)
    meas = pic.growth_rate(h.t, h.energy[:, 1])
    pred = pic.predicted(w, kmod=kmod, aliases=pic.ALL_ALIASES)
    print(f"{w.dt} kc={w.filt_kc} l={w.shape_order} kmod={kmod}: measured {meas:.4f} predicted {pred[0]:.4f} "
          f"at k = ({pred[1]:.2f}, {pred[2]:.2f}) alias {pred[3]}  ({h.seconds:.1f} s)")
    return h, meas, pred[0]


def test_unfiltered_run_grows_at_the_predicted_rate():
    need_gpu()
    hyb_module()
    from paper_1502_01376_gb300 import pic
    h, meas, pred = _case(pic.TABLE1, 2000)
    assert meas > 0.1                                       # the (0, +-1) NCI, clearly
    assert LO * pred <= meas <= HI * pred


def test_filter_leaves_the_zero_zero_modes_and_a_smaller_step_slows_them():
    need_gpu()
    hyb_module()
    from paper_1502_01376_gb300 import pic
    w = pic.TABLE1.scaled(filt_kc=0.5)
    _, m08, p08 = _case(w, 6000)
    _, m04, p04 = _case(w.scaled(dt=0.04), 12000)
    assert LO * p08 <= m08 <= HI * p08
    assert LO * p04 <= m04 <= HI * p04
    assert m04 < 0.6 * m08                                   # Sec. 4: a smaller dt lowers the (0, 0) growth


def test_k1_modification_removes_the_zero_zero_modes():
    """Fig. 3b: with the printed modification the E2 energy stays at its noise level where the
    unmodified run grows by orders of magnitude; later the (+-1, +-2) modes grow with quadratic
    shapes (no faster than predicted), and with cubic shapes nothing grows."""
    need_gpu()
    hyb_module()
    from paper_1502_01376_gb300 import pic
    w = pic.TABLE1.scaled(filt_kc=0.5)
    h0, _, _ = _case(w, 3500)
    h2, m2, p2 = _case(w, 8000, kmod=pic.BUMP)
    h3, m3, p3 = _case(w.scaled(shape_order=3), 8000, kmod=pic.BUMP)

    def at(h, t):
        return h.energy[np.searchsorted(h.t, t), 1]
    noise = at(h2, 40.0)
    assert at(h0, 280.0) > 1e5 * at(h0, 40.0)               # without: (0, 0) growth
    assert at(h2, 280.0) < 10.0 * noise                      # with: none over the same time
    assert m2 <= HI * p2 + 2e-3                              # the later (+-1, +-2) growth
    assert h3.energy[-1, 1] < 10.0 * at(h3, 40.0)           # cubic shapes: flat to t = 640
    assert m3 <= HI * p3 + 2e-3
