"""Write tests/golden/band_sizes.txt: |B| and |G| of the oracle's band for the
benchmark and parity workloads (calls only oracle/)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle.band import build_band  # noqa: E402
from oracle.geometry import sphere, torus  # noqa: E402

CASES = [("sphere", (), 256), ("sphere", (), 128), ("torus", (1.0, 0.4), 128)]

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "band_sizes.txt")
    with open(out, "w") as fh:
        fh.write("# |B| and |G| of the tube band (lambda^2 = 17) on [-2,2]^3, written by make_band_sizes.py\n")
        fh.write("# columns: surface params 1/dx n_band n_ghost\n")
        for kind, params, inv in CASES:
            surf = sphere(*params) if kind == "sphere" else torus(*params)
            b = build_band(surf, 1.0 / inv)
            fh.write(f"{kind} {','.join(map(str, params)) or '-'} {inv} {b.nb} {b.ng}\n")
            fh.flush()
            print(kind, inv, b.nb, b.ng, flush=True)
