"""Precision study of the decode paths against the FP64 oracle (needs a GB300).

    python tests/precision_study.py

For the small map (64 x 64 cells, one tile) at D = 1024, 4096, 8192 and 16384,
and for the first 20 scans of the paper-scale map (400 x 400 cells, 4 x 4
tiles, D = 8192), runs the whole path through the C ABI with each decode
precision and prints, per case and path, the normwise error of the raw class
maps P and of the normalised maps P_hat, and the largest absolute error of
Pr(psi = 1), all against the oracle's pipeline (Eq. loc-query through Eq.
softmax) on the same seeded inputs.  The parity tests hold these errors to the
tolerances; this prints the values themselves, as a Markdown table.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from helpers import config_for, normwise, oracle_grid, run_gpu  # noqa: E402
from paper_2408_09066_gb300 import build, synth  # noqa: E402
from paper_2408_09066_gb300 import vsaogm as V  # noqa: E402

PATHS = [("FP32 SIMT", V.DECODE_FP32), ("BF16x3", V.DECODE_BF16X3),
         ("FP16x3", V.DECODE_FP16X3), ("FP8x3", V.DECODE_FP8X3)]


def oracle_pipeline(cfg, xy, labels):
    g = oracle_grid(cfg)
    nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
    return oracle.pipeline(g, nx, ny, xy, labels, cfg.r_occ, cfg.r_emp, cfg.rho, "tile")


def errors(wl, prec, want):
    got = run_gpu(config_for(wl, decode_prec=prec), wl.xy, wl.labels)
    return (normwise(got["P"], want["P"]), normwise(got["Phat"], want["Phat"]),
            float(np.abs(got["occ"] - want["pr1"]).max()))


def main():
    build.build()
    cases = [(f"small map, D = {D}", synth.small_scan(D=D), PATHS[1:])
             for D in (1024, 4096, 8192, 16384)]
    cases.append(("paper map (first 20 scans), D = 8192", synth.paper_trajectory(n_scans=20),
                  PATHS))
    print("| case | " + " | ".join(name for name, _ in PATHS) + " |")
    print("|---|" + "---|" * len(PATHS))
    for label, wl, paths in cases:
        want = oracle_pipeline(config_for(wl), wl.xy, wl.labels)
        cells = {}
        for name, prec in paths:
            p, ph, pr = errors(wl, prec, want)
            cells[name] = f"{p:.1e} / {ph:.1e} / {pr:.1e}"
        print(f"| {label} | " + " | ".join(cells.get(name, "—") for name, _ in PATHS) + " |")
    print("\n(normwise P / normwise P_hat / max |dPr(psi=1)|)")


if __name__ == "__main__":
    main()
