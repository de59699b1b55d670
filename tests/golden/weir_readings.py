"""Record which readings decide the failure of the sharp-crested weir
(Section 5.5; finding F5 of the design notes): the FP64 oracle runs the
weir at CFL 0.45 with each alternative reading switched on (orc_run_record's
experiment bits) until its first non-admissible step, and the time reached is
written to a text record.

    python tests/golden/weir_readings.py NX NY T_STOP VARIANT[,VARIANT...] OUT

VARIANT is one of: default, bj_printed, no_pos, bj_printed+no_pos, aE_one,
aE_two_layer.  Calls only oracle/ (and the input generator cases.weir_e5).
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_1806_04960_gb300 import cases  # noqa: E402

VARIANTS = {
    "default": {},
    "bj_printed": {"bj_printed": True},
    "no_pos": {"no_pos": True},
    "bj_printed+no_pos": {"bj_printed": True, "no_pos": True},
    "aE_one": {"aE_mode": 1},
    "aE_two_layer": {"aE_mode": 2},
}


def first_failure(c, kw, t_stop, chunk=50):
    """(time reached, steps, failed?) of the oracle's run with switches kw."""
    q, t, steps = c.q, 0.0, 0
    while t < t_stop:
        try:
            q2, dts, _, _ = oracle.run_record(c, chunk, [0], q=q, cfl=c.cfl, **kw)
        except oracle.OracleError:
            for k in range(1, chunk + 1):
                try:
                    _, dts, _, _ = oracle.run_record(c, k, [0], q=q, cfl=c.cfl, **kw)
                except oracle.OracleError:
                    return t + (float(dts.sum()) if k > 1 else 0.0), steps + k, True
            return t, steps, True
        q, t, steps = q2, t + float(dts.sum()), steps + chunk
    return t, steps, False


def main(argv):
    nx, ny, t_stop = int(argv[1]), int(argv[2]), float(argv[3])
    names, out = argv[4].split(","), argv[5]
    c = cases.weir_e5(nx, ny)
    rows = []
    for name in names:
        t0 = time.perf_counter()
        t, steps, failed = first_failure(c, VARIANTS[name], t_stop)
        rows.append((name, t, steps, failed, time.perf_counter() - t0))
        print(rows[-1], flush=True)
    new = not os.path.exists(out)
    with open(out, "a") as f:
        if new:
            f.write("# Weir of Section 5.5 (cases.weir_e5), FP64 oracle, CFL 0.45: time reached by\n"
                    "# each reading variant (failed = 1: the next step is non-admissible; 0: stopped\n"
                    "# at T_STOP).  Written by tests/golden/weir_readings.py.\n"
                    "# columns: nx ny variant t_reached steps failed\n")
        for name, t, steps, failed, _ in rows:
            f.write(f"{nx} {ny} {name} {t:.6f} {steps} {int(failed)}\n")


if __name__ == "__main__":
    main(sys.argv)
