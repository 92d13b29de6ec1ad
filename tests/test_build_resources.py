"""Static resource checks of the CUDA kernels from the compiler's own report (nvcc -Xptxas -v for
sm_103a; no GPU needed).  No kernel spills registers to local memory except three whose small
spills are measured and accepted: the per-atom pair kernel at 201 and 208 q per pass (it runs at
the 255-register cap; passes of ~101 q without spills were slower) and the plain bfloat16 GEMM
used for the surrogate's narrow shapes."""
import concurrent.futures as cf
import glob
import os
import re
import shutil
import subprocess

import pytest

from paper_1306_2258_gb300 import build

# mangled-name fragment -> (largest accepted spill stores, spill loads) in bytes
ACCEPTED = {
    "k_debye_atomic_pairs2ILi52ELi101E": (80, 96),
    "k_debye_atomic_pairs2ILi52ELi104E": (56, 72),
    "k_gemm_tn": (28, 28),
}


def _report(src, out_dir):
    obj = os.path.join(out_dir, os.path.basename(src) + ".o")
    r = subprocess.run([build.NVCC, *build.ARCH, *build.FLAGS, "-Xptxas=-v", "-c", src, "-o", obj],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    rows, name = [], None
    for line in r.stderr.splitlines():
        m = re.search(r"Function properties for (\S+)", line)
        if m:
            name = m.group(1)
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and name:
            rows.append((name, int(m.group(1)), int(m.group(2))))
            name = None
    return rows


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    if not (os.path.exists(build.NVCC) or shutil.which(build.NVCC)):
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("ptxas"))
    srcs = sorted(glob.glob(os.path.join(build.CSRC, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        return [row for rows in ex.map(lambda s: _report(s, out), srcs) for row in rows]


def test_every_kernel_reported(report):
    names = [n for n, _, _ in report]
    for k in ("k_debye_mixed_pairs2", "k_debye_mixed", "k_debye_fp64", "k_debye_adjoint", "k_debye_atomic_pairs2",
              "k_quad_amp", "k_pair_histogram", "k_gemm_tcp", "k_adjoint_gather", "k_reduce_segments_fix"):
        assert any(k in n for n in names), k


def test_no_register_spills_beyond_the_accepted_ones(report):
    for name, st, ld in report:
        if st == 0 and ld == 0:
            continue
        limit = next((v for k, v in ACCEPTED.items() if k in name), None)
        assert limit is not None, f"{name} spills {st} B stores / {ld} B loads"
        assert st <= limit[0] and ld <= limit[1], (name, st, ld)
