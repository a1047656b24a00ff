"""Time operator evaluations of one solver: ``python -m paper_2110_13735_gb300.evalbench --N 64``.

Creates a 2-D solver on the bosonic Gaussian of mass 5 and temperature 0.5 (Maxwell molecules,
R = 6, T = (3 + sqrt 2) R / 2), runs ``--warmup`` untimed and ``--evals`` timed evaluations of
Q_eps through the C ABI and prints one JSON line: the kernel configuration, the operator kernel's
time per launch (CUDA events recorded by the library around it) and the Q_{1,q} terms and FP32 or
FP64 FMA rate that this time gives (4 flops per term).  Used to profile one operator size alone.
"""
from __future__ import annotations

import argparse
import json

from . import bn, inputs


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--N", type=int, default=64)
    ap.add_argument("--eps", type=float, default=1.0)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--kernel", choices=["maxwell", "hard_sphere"], default="maxwell")
    ap.add_argument("--evals", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    args = ap.parse_args(argv)
    bn.load()
    R = 6.0
    T = inputs.box_half_width(R)
    prec = bn.MIXED if args.precision == "mixed" else bn.FP64
    kern = bn.MAXWELL if args.kernel == "maxwell" else bn.HARD_SPHERE
    with bn.Solver(2, args.N, T, R, kern, args.eps, precision=prec) as s:
        s.set_state(inputs.gaussian(2, args.N, T, 5.0, 0.5))
        for _ in range(args.warmup):
            s.eval_collision()
        s.profile_enable(True)
        s.profile_read()
        for _ in range(args.evals):
            s.eval_collision()
        ev_ms, n, span_ms, ns = s.profile_read()
        cfg = s.kernel_config()
    terms = (2.0 * (args.N ** 3 - args.N) / 3.0) ** 2 if args.eps != 0.0 else 0.0
    ms = ev_ms / max(n, 1)
    print(json.dumps({"N": args.N, "eps": args.eps, "precision": args.precision, "kernel": args.kernel,
                      "kernel_config": cfg, "ms_per_launch": ms, "launches": n,
                      "q1q_terms": terms, "tflops": 4.0 * terms / (ms * 1e-3) / 1e12 if ms > 0 else None}))


if __name__ == "__main__":
    main()
