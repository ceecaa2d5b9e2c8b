"""Write c1_freeze_oracle.json: the FP64 oracle's freezing history of the 128x64
sessile ferrofluid drop (R = 24, vertical field, Bo_m = 0.5, chi = 1, Ste = 0.1)
run until Q_L first reaches 0.99.

Q_L is Eq. 51 (solid fraction of the droplet cells C >= 1/2); t_freeze is the
first time with Q_L >= 0.99, linear in time between steps.  Only the oracle is
called, so the stored values are independent of the CUDA path.

    python tests/golden/make_c1_freeze.py [threads]
"""
import json
import os
import sys
import time

_ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, _ROOT)

import oracle  # noqa: E402
from paper_2511_10257_gb300 import inputs as I  # noqa: E402

CHUNK = 500
MAX_STEPS = 60000


def main(threads: int) -> None:
    case = I.config_small()
    o = oracle.Oracle(case, threads=threads)
    t0 = time.time()
    history = []
    n = 0
    while n < MAX_STEPS:
        o.step(CHUNK)
        n += CHUNK
        s = o.stats()
        history.append([n, s["Q_L"]])
        print(f"step {n} Q_L {s['Q_L']:.6f} ({time.time() - t0:.0f} s)", flush=True)
        if s["t_freeze"] >= 0.0:
            break
    s = o.stats()
    out = {
        "what": "FP64 oracle, 128x64 sessile drop R=24, vertical field, Bo_m=0.5, chi=1, "
                "Ste=0.1; Q_L by Eq. 51, t_freeze = first t with Q_L >= 0.99",
        "dt": case["dt"],
        "steps": n,
        "t_freeze": s["t_freeze"],
        "final": {k: s[k] for k in ("sum_C", "sum_He", "Q_L", "t")},
        "Q_L_every_500_steps": history,
        "oracle_threads": threads,
        "wall_s": round(time.time() - t0, 1),
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_freeze_oracle.json"),
              "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count() or 1)
