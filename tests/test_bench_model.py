"""bench.py's work model covers every kernel the library can report: each name of the kernel-name table in
csrc/lgf.cu, in both precisions and for a power-of-two and a mixed-radix lattice, has a positive
algorithmic byte count and a known arithmetic kind. CPU only."""
import pathlib
import re

import bench


def kernel_names():
    src = (pathlib.Path(__file__).resolve().parents[1] / "paper_1210_8018_gb300" / "csrc" / "lgf.cu").read_text()
    table = re.search(r"kKernelBase\[KID_COUNT\]\s*=\s*\{(.*?)\};", src, re.S)
    return re.findall(r'"([a-z0-9_]+)"', table.group(1))


def test_every_reported_kernel_has_a_work_model():
    names = kernel_names()
    assert len(names) == len(set(names)) >= 20
    for name in names:
        for prec in ("f32", "f64"):
            for dims in [(64, 64, 64, 64), (6, 4, 8, 10)]:
                b, f, kind = bench.algorithmic(name + "." + prec, dims)
                assert b > 0 and f >= 0 and kind in (None, "fp32", "fp64"), (name, prec, b, f, kind)
                if kind:
                    assert f > 0, (name, prec)
