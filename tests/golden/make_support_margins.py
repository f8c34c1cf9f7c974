"""Write support_margins.txt: for every operator of the measured workloads,
the support radius, the radius the oracle's threshold guard keeps, and the
smallest relative distance |u - u_s| / u_s of any pixel pair from the
coupling threshold.  Calls the oracle only.

    python tests/golden/make_support_margins.py
"""
from pathlib import Path
import sys

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import oracle as O  # noqa: E402
from paper_1504_04653_gb300 import workloads as W  # noqa: E402


def main():
    out = ["# workload op lmax r_s(hex) r_used(hex) margin",
           "# r_used = r_s unless a pair lies within 1e-12 (relative) of the threshold"]
    grids = {}
    for key in ("lmax64", "lmax500", "lmax1500", "lmax3000", "batched32"):
        wl = W.WORKLOADS[key]
        g = grids.setdefault(wl.lmax, O.grid(wl.lmax))
        for op, r_s in enumerate(wl.radii()):
            r, m = O.guarded_radius(g, float(r_s))
            out.append(f"{key} {op} {wl.lmax} {float(r_s).hex()} {r.hex()} {m:.12e}")
            print(out[-1], flush=True)
    (Path(__file__).resolve().parent / "support_margins.txt").write_text("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
