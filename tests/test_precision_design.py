"""Why the float32 path has no float64 island for E - |m|^2/(2 rho).

The energy balance (Sec. 2.4, reading s11) takes e = E - K (K = |m|^2/(2 rho))
when that is at least eta E.  In a cold, fast flow near the switch (Mach ~ 40
here, where E - K is ~1e-3 of E) this is a difference of numbers a thousand
times larger, and a float32 state loses about 1e-4 of e there.  A float64
island for that subtraction would have to protect it from the rounding of
everything K is made of: this test evaluates the oracle's own step on float32
arrays (its arithmetic is dtype-generic numpy) and shows
  * all-float32: e is off by more than 1e-4 (relative L1, 10 steps);
  * E and the energy tensor nE kept in float64 (the island): the error stays
    within a factor 2 of the all-float32 one -- rho and m are still float32;
  * every conserved field kept in float64: the error drops below 1e-6.
The GPU float32 path shows the same behaviour (test_gpu_balance.py).
"""
import numpy as np

import oracle as O
from helpers import cold_flow_state, rel_l1

WIDE_ISLAND = ("E", "nExx", "nEyy", "nEzz", "nExy", "nExz", "nEyz")
WIDE_ALL = ("rho", "mx", "my", "mz", "E", "n", "qx", "qy", "qz") + WIDE_ISLAND[1:]


def run_mixed(st0, prm, steps, wide):
    """``steps`` oracle steps with the fields in ``wide`` stored in float64 and the
    rest in float32 (potential and step size from the float64 run)."""
    ref = st0
    st = {f: (v if f in wide else v.astype(np.float32)) for f, v in st0.items()}
    for _ in range(steps):
        dt = O.cfl_dt(ref, prm)
        phi = O.solve_poisson(ref, prm)
        ref, _ = O.advance(ref, phi, dt, prm)
        st, _ = O.advance(st, phi.astype(np.float32), np.float32(dt), prm)
        st = {f: (v.astype(np.float64) if f in wide else v.astype(np.float32)) for f, v in st.items()}
    return st, ref


def test_float64_island_does_not_protect_the_switch():
    st0, h = cold_flow_state(24, 40)
    prm = O.Params(h=h)
    errs = {}
    for name, wide in (("f32", ()), ("island", WIDE_ISLAND), ("all", WIDE_ALL)):
        st, ref = run_mixed(st0, prm, 10, wide)
        assert st["rho"].dtype == (np.float64 if "rho" in wide else np.float32)
        errs[name] = rel_l1(st["e"], ref["e"])
    assert errs["f32"] > 1e-4, errs
    assert errs["island"] > 0.5 * errs["f32"], errs
    assert errs["all"] < 1e-6, errs
