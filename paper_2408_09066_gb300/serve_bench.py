"""Serving benchmark: 32 robots with resident maps (256^2 to 1024^2 cells, D = 8192,
tiles of 128 cells), Poisson arrivals of scan updates (1080 beams x 21 points)
and window queries (128^2 to 512^2 cells), swept in rate until the server
saturates.  Prints one JSON line per rate with p50/p99 latency per request kind
and the achieved throughput.

    python -m paper_2408_09066_gb300.serve_bench [--robots 32] [--duration 2]
        [--deadline-ms T]   # drop requests not started T ms after arrival
"""
from __future__ import annotations

import argparse
import json

from . import serving, synth
from . import vsaogm as V


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--robots", type=int, default=32)
    p.add_argument("--slots", type=int, default=8)
    p.add_argument("--duration", type=float, default=2.0)
    p.add_argument("--rates", type=str, default="250,500,1000,2000,4000,8000")
    p.add_argument("--query-frac", type=float, default=0.5)
    p.add_argument("--decode", choices=["bf16x3", "fp16x3", "fp32"], default="bf16x3")
    p.add_argument("--deadline-ms", type=float, default=None,
                   help="start deadline per request; later requests are dropped as expired")
    a = p.parse_args()
    prec = {"fp32": V.DECODE_FP32, "bf16x3": V.DECODE_BF16X3, "fp16x3": V.DECODE_FP16X3}[a.decode]
    fleet = synth.robot_fleet(a.robots)
    cfgs = serving.fleet_configs(fleet, D=8192, decode_prec=prec)
    max_points = max(len(s[1]) for r in fleet for s in r.scans)
    srv = serving.Server(cfgs, max_points=max_points, max_window=512, n_slots=a.slots)
    try:
        # warm-up: closed batches touching every robot with both request kinds,
        # so no measured request pays for a first launch of a kernel
        srv.run(serving.poisson_requests(fleet, 2000.0, 0.5, a.query_frac, seed=99),
                realtime=False)
        for i, rate in enumerate(float(x) for x in a.rates.split(",")):
            deadline = None if a.deadline_ms is None else a.deadline_ms / 1e3
            reqs = serving.poisson_requests(fleet, rate, a.duration, a.query_frac, seed=i,
                                            deadline=deadline)
            done = srv.run(reqs, realtime=True)
            s = serving.summarize(done, a.duration)
            s.update({"offered_per_s": rate, "robots": a.robots, "slots": srv.n_slots,
                      "decode": a.decode, "D": 8192, "deadline_ms": a.deadline_ms,
                      "saturated": s["requests_per_s"] < 0.9 * rate})
            print(json.dumps(s), flush=True)
    finally:
        srv.close()


if __name__ == "__main__":
    main()
