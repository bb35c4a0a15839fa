"""A C99 program linked against libpic_gb300.so alone drives the hot path
on the GPU: pic_create, pic_sample_mms, pic_step, pic_mms_error and
pic_get_stats, in both forms, on the legacy default stream with the
library's own cudaMalloc. Its error norms and counters equal, bit for bit,
those of the same run through the Python binding (torch allocator and
stream): the boundary carries no hidden state."""
import ctypes
import shutil
import subprocess

import numpy as np
import pytest

from paper_2602_15130_gb300 import Pic, _lib

pytestmark = pytest.mark.gpu

PROGRAM = r"""#include <stdio.h>
#include <stdlib.h>
#include "pic.h"
static int run(int precision) {
  pic_config c;
  pic_config_default(&c);               /* 8^3 cells, 4096 particles, K = 16 */
  c.precision = precision;
  c.cg_tol = precision == PIC_MIXED ? 1e-6 : 1e-10;
  pic_ctx* ctx = NULL;
  pic_status s = pic_create(&c, NULL, NULL, &ctx);
  if (s != PIC_OK) { printf("create %s\n", pic_status_string(s)); return 1; }
  if ((s = pic_sample_mms(ctx, 0.0)) != PIC_OK) { printf("sample %s\n", pic_status_string(s)); return 2; }
  if ((s = pic_step(ctx, 3)) != PIC_OK) { printf("step %s\n", pic_status_string(s)); return 3; }
  pic_errors e;
  pic_stats st;
  if (pic_mms_error(ctx, &e) != PIC_OK || pic_get_stats(ctx, &st) != PIC_OK) return 4;
  printf("%d", precision);
  for (int q = 0; q < 7; ++q) printf(" %.17g %.17g", e.eps2[q], e.epsinf[q]);
  printf(" %lld %lld %d\n", (long long)st.n_cand, (long long)st.n_coll, (int)st.cg_iters_last);
  pic_destroy(ctx);
  return 0;
}
int main(void) { return run(PIC_FP64) || run(PIC_MIXED); }
"""


def test_c_program_steps_on_the_gpu_like_the_binding(tmp_path):
    cc = shutil.which("gcc")
    if not cc:
        pytest.skip("no host C compiler")
    import __graft_entry__ as g

    g.build()
    src = tmp_path / "drive.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "drive"
    lib = _lib.LIB_PATH
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", str(_lib.HEADER.parent), str(src), "-o", str(exe),
                    "-L", str(lib.parent), "-lpic_gb300", f"-Wl,-rpath,{lib.parent}"], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    rows = [line.split() for line in r.stdout.splitlines()]
    assert [int(row[0]) for row in rows] == [0, 1]
    L = _lib.load()
    for row in rows:
        cfg = _lib.PicConfig()
        assert L.pic_config_default(ctypes.byref(cfg)) == _lib.PIC_OK
        cfg.precision = int(row[0])
        cfg.cg_tol = 1e-6 if cfg.precision == _lib.PIC_MIXED else 1e-10
        sim = Pic(cfg)
        sim.sample_mms(0.0)
        sim.step(3)
        e = sim.mms_error()
        st = sim.stats()
        sim.close()
        want = []
        for q in ("x", "y", "z", "u", "v", "w", "phi"):
            want += [e["eps2"][q], e["epsinf"][q]]
        got = [float(t) for t in row[1:15]]
        assert np.array_equal(np.array(got), np.array(want)), (row[0], got, want)
        assert [int(row[15]), int(row[16]), int(row[17])] == [st["n_cand"], st["n_coll"], st["cg_iters_last"]]
        assert st["n_coll"] > 0
