"""The no-allocation diagnostics entry point against the handle's diagnostics.

flic_state_diagnostics_noalloc serves callers that cannot allocate device
memory (the device memory is reserved by another owner, or an allocation's
implicit synchronisation is not acceptable); its scratch is a file-scope device
array shared by all calls.  It must give what flic_diagnostics gives for the
same state, on consecutive calls (the shared scratch keeps the previous call's
contents).  This file is collected last.
"""
import numpy as np
import pytest

from paper_1311_0861_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_1311_0861_gb300 import flic
    if not os.path.exists(flic.LIB_PATH):
        from paper_1311_0861_gb300 import build
        build.build()
    flic.load()
    return torch, flic


KEYS = ("mass_gas", "mass_bme", "mom_x", "mom_y", "mom_z", "ekin_gas", "eint_gas", "ekin_bme", "etherm_bme",
        "epot", "kappa_gas", "kappa_bme")


def test_noalloc_matches_handle_diagnostics_on_two_calls(env):
    torch, flic = env
    N = 24
    s = I.random_state((N, N, N), seed=11)
    with flic.Grid(N, precision="fp64", box=(-1.0, -1.0 + N * s.h), gamma=s.gamma) as g:
        g.set_state(s.state)
        ref = g.diagnostics()
        phi = g.solve_poisson()
    dev = [torch.from_numpy(np.ascontiguousarray(s.state[f])).cuda() for f in flic.FIELDS]
    phid = torch.from_numpy(phi).cuda()
    torch.cuda.synchronize()
    for _ in range(2):
        d = flic.state_diagnostics_noalloc(dev, phid, N, s.h, s.gamma)
        for k in KEYS:
            assert abs(d[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (k, d[k], ref[k])
        assert abs(d["vmax"] - ref["vmax"]) <= 1e-14 * ref["vmax"]
        assert d["status"] == 0 and not d["nonphysical"]


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    """The C entry point itself refuses a grid larger than its scratch is built for
    (the check runs before any device work)."""
    import ctypes
    torch, flic = env
    lib = flic.load()
    dev = [torch.zeros(8, dtype=torch.float64, device="cuda") for _ in range(22)]
    ptrs = (ctypes.c_void_p * 22)(*[t.data_ptr() for t in dev])
    out = flic.Diag()
    rc = lib.flic_state_diagnostics_noalloc(ptrs, None, 2048, 0.01, 5.0 / 3.0, None, ctypes.byref(out))
    assert rc == flic.ERR_INVALID_ARG
    assert b"1024" in lib.flic_last_error(None)


NOALLOC_FIRST_CALL = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1311_0861_gb300 import flic, inputs as I
import oracle as O
N = 16
s = I.random_state((N, N, N), seed=21)
dev = [torch.from_numpy(np.ascontiguousarray(s.state[f])).cuda() for f in flic.FIELDS]
torch.cuda.synchronize()
d = flic.state_diagnostics_noalloc(dev, None, N, s.h, s.gamma)   # the library's first call in this process
prm = O.Params(h=s.h, gamma=s.gamma)
ref = O.diagnostics(s.state, np.zeros((N, N, N)), prm)
ref["vmax"] = O.max_signal_speed(s.state, prm)
print(json.dumps({"got": {k: d[k] for k in ref}, "want": ref}))
"""


def test_noalloc_as_the_first_call_in_a_fresh_process(env):
    """The entry point's set-up (module load, address look-up) on a device where
    no other call of the library ran first; checked against the oracle's sums."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", NOALLOC_FIRST_CALL, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    for k, want in out["want"].items():
        got = out["got"][k]
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (k, got, want)
