"""Count the wide components of each workload recipe (test infrastructure).

A component is wide when, along a periodic axis, the minimum-image
displacements of its sites from its first site span half the period or more
(``oracle.wide_components``); its centroid is then a convention rather than
the centre of a blob. This prints the counts on seeded samples of each
recipe, using only the oracle and the seeded input generators:

    python -m oracle.wide_report
"""
from __future__ import annotations

from paper_1607_00908_gb300 import inputs as I

from . import detect as O


def count(F) -> tuple[int, int]:
    lab, K = O.label_components(O.foreground(F))
    return K, int(O.wide_components(lab, K).sum())


def main() -> None:
    c0 = [count(F) for seed in range(1, 9) for F in I.workload_c0(seed)]
    print("128^2 smoothed noise sigma 3, seeds 1-8, both frames (K, wide):", c0)
    c1 = [count(F) for k, F in enumerate(I.workload_c1(1, 64)) if k % 8 == 0]
    print("1024^2 smoothed noise sigma 4, seed 1, every 8th frame (K, wide):", c1)
    F = next(iter(I.workload_c2(1, 1)))[0]
    print("4096^2 RSA discs, seed 1, frame 0 (K, wide):", count(F))
    c3 = [count(I.smoothed_noise(L, L, sig, s)) for L, sig, s in I.batch_instances()]
    print("batched instances, first frames: %d of %d with a wide component, %d wide in all"
          % (sum(w > 0 for _, w in c3), len(c3), sum(w for _, w in c3)))
    c4 = [count(I.smoothed_noise(L, L, 4.0, s)) for L, rec, s in I.serve_sims() if rec == "noise"]
    print("served smoothed-noise sims, first frames: %d wide in %d sims (disc sims: radii <= 12, never wide)"
          % (sum(w for _, w in c4), len(c4)))


if __name__ == "__main__":
    main()
