"""The debug build (librgf_debug.so, -DRGF_DEBUG): device-side checks of the
indices kernels take from data (Gauss-Jordan pivot rows, the server's slot
table) stay silent on correct runs at small and odd block sizes, and the
arithmetic is that of the normal build.

The debug library runs in a child process (RGF_DEBUG_LIB=1 selects it at
import); the parent runs the same work with the normal library.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORK = r'''
import json
import numpy as np
from paper_2609_37058_b300 import rgf
from synth import random_device
from synth.devices import energy_grid, uneven_batch

def run():
    out = {}
    for b in (1, 2, 3, 8):
        dev = random_device(5, b, 300 + b, metal_frac=0.25, gap_offset=0.6)
        E = energy_grid(-1.5, 1.5, 9)
        for prec, tag in ((rgf.RGF_MIXED, "mixed"), (rgf.RGF_FP64, "fp64")):
            with rgf.Plan(5, b, precision=prec, eta=1e-5) as p:
                p.set_device(dev)
                T, err, fl = p.transmission(E)
            out[f"{tag}{b}"] = T.tolist()
    jobs = uneven_batch(6, 9, N_lo=3, N_hi=9, b_choices=[1, 2, 3, 8], n_E=5, eta=1e-5)
    with rgf.Server(slots=8, class_step=8) as sv:
        tickets = [sv.submit(d, E, eta) for d, E, eta in jobs]
        res = [sv.poll(t, timeout_us=300_000_000) for t in tickets]
    out["server"] = [r[0].tolist() for r in res]
    return out
'''


@pytest.fixture(scope="module")
def libs():
    from paper_2609_37058_b300 import build
    build.build()
    build.build(debug=True)


def test_debug_build_is_silent_and_matches(libs):
    child = WORK + r'''
out = run()
L = rgf.lib()
out["debug_build"] = int(L.rgf_debug_build())
out["flags"] = int(L.rgf_debug_flags())
print("RESULT " + json.dumps(out))
'''
    env = dict(os.environ, RGF_DEBUG_LIB="1")
    p = subprocess.run([sys.executable, "-c", child], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    line = [x for x in p.stdout.splitlines() if x.startswith("RESULT ")][-1]
    dbg = json.loads(line[len("RESULT "):])
    assert dbg["debug_build"] == 1
    assert dbg["flags"] == 0

    ns = {}
    exec(WORK, ns)
    from paper_2609_37058_b300 import rgf
    assert rgf.lib().rgf_debug_build() == 0 and rgf.lib().rgf_debug_flags() == 0
    rel = ns["run"]()
    for key, T in rel.items():
        if key == "server":
            for a, b in zip(T, dbg[key]):
                assert np.abs(np.array(a) - np.array(b)).max() <= 1e-12
        else:
            assert np.abs(np.array(T) - np.array(dbg[key])).max() <= 1e-12, key
