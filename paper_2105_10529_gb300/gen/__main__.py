"""Write the generated matrix-element headers into csrc/generated/.

    python -m paper_2105_10529_gb300.gen
"""
import os
from fractions import Fraction

from . import bg_tables, qcd_diagrams, qq_processes, rc_tables

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "csrc", "generated")

PROCESSES = [
    (2, "gg_tt", Fraction(1)),
    (3, "gg_ttg", Fraction(1)),
    (4, "gg_ttgg", Fraction(1, 2)),
]


def write_all(out_dir: str = OUT) -> list:
    os.makedirs(out_dir, exist_ok=True)
    written = []
    items = [(f"me_{name}.cuh", lambda k=k, name=name, sym=sym: qcd_diagrams.generate_gluon_process(k, name, sym)[0])
             for k, name, sym in PROCESSES]
    items += [("me_uu_tt.cuh", lambda: qq_processes.generate_uu_tt()[0]),
              ("me_ug_ttu.cuh", lambda: qq_processes.generate_ug_ttu()[0]),
              ("bg_gg_ttggg.cuh", lambda: bg_tables.generate(5, "gg_ttggg")[0])]
    # the recursion's tables of the lighter gluon processes (their derivatives run the reverse sweep)
    items += [(f"bg_{name}.cuh", lambda k=k, name=name: bg_tables.generate(k, name)[0])
              for k, name in ((2, "gg_tt"), (3, "gg_ttg"), (4, "gg_ttgg"))]
    # the helicity-recycled recursion of g g -> t tbar g g (warp-per-event schedule 4)
    items += [("rc_gg_ttgg.cuh", lambda: rc_tables.generate("gg_ttgg")[0])]
    for fname, make in items:
        src = make()
        path = os.path.join(out_dir, fname)
        old = open(path).read() if os.path.exists(path) else None
        if old != src:
            with open(path, "w") as f:
                f.write(src)
        written.append(path)
    return written


if __name__ == "__main__":
    for p in write_all():
        print(p)
