"""Write batched_replicates.txt: the replicate list of the batched
refinement study (256 replicates, host generator seed 42), one line per
replicate: index, mesh edge n, particles, K, Philox seed, sigma0.

    python tests/golden/write_batched_replicates.py
"""
from pathlib import Path
import sys

sys.path.insert(0, str(Path(__file__).resolve().parents[2]))

from paper_2602_15130_gb300 import workloads  # noqa: E402


def lines():
    yield "# r n n_particles K seed sigma0  (workloads.batched(256, seed=42))"
    for r, p in enumerate(workloads.batched()):
        yield f"{r} {p['n']} {p['n_particles']} {p['K']} {p['seed']} {p['sigma0']:.17g}"


if __name__ == "__main__":
    out = Path(__file__).with_name("batched_replicates.txt")
    out.write_text("\n".join(lines()) + "\n")
    print(out)
