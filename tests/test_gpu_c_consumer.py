"""The C ABI used from C, with no Python in the process: a program compiled
with gcc against include/dfpr.h and linked to libdfpr.so reads a graph and a
batch from files, runs Static, applies the batch, tunes the sweep, runs DF-P
with the loop on the host and then on the device, and writes the ranks.  The
ranks must equal the oracle's within 1e-9 and the two loops must agree bit
for bit."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = 1e-9

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "dfpr.h"

static void* slurp(const char* path, size_t* bytes) {
  FILE* f = fopen(path, "rb");
  if (!f) return NULL;
  fseek(f, 0, SEEK_END);
  long len = ftell(f);
  fseek(f, 0, SEEK_SET);
  void* p = malloc(len > 0 ? (size_t)len : 1);
  if (p && len > 0 && fread(p, 1, (size_t)len, f) != (size_t)len) { free(p); p = NULL; }
  fclose(f);
  *bytes = (size_t)len;
  return p;
}

#define CHECK(call) do { pr_status s_ = (call); if (s_ != PR_OK) { \
  fprintf(stderr, "%s failed: %s %s\n", #call, pr_status_string(s_), pr_last_error(g)); return 1; } } while (0)

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  const char* dir = argv[1];
  char path[4096];
  size_t nb, ob, cb, bb;
  snprintf(path, sizeof path, "%s/n.bin", dir);
  int32_t* np_ = (int32_t*)slurp(path, &nb);
  snprintf(path, sizeof path, "%s/off.bin", dir);
  int64_t* off = (int64_t*)slurp(path, &ob);
  snprintf(path, sizeof path, "%s/col.bin", dir);
  int32_t* col = (int32_t*)slurp(path, &cb);
  snprintf(path, sizeof path, "%s/batch.bin", dir);   /* n_del, n_ins, then del_src, del_dst, ins_src, ins_dst */
  int32_t* b = (int32_t*)slurp(path, &bb);
  if (!np_ || !off || !col || !b) return 3;
  const int32_t n = np_[0];
  const int64_t m = off[n];
  const int32_t nd = b[0], ni = b[1];
  const int32_t *ds = b + 2, *dd = ds + nd, *is = dd + nd, *id = is + ni;
  pr_graph* g = NULL;
  CHECK(pr_graph_create(n, m, off, col, NULL, &g));
  pr_stats st;
  CHECK(pr_update(g, PR_STATIC, 0.85, 1e-10, NULL, &st));
  double* r0 = (double*)malloc(sizeof(double) * n);
  double* r1 = (double*)malloc(sizeof(double) * n);
  double* r2 = (double*)malloc(sizeof(double) * n);
  CHECK(pr_ranks(g, r0));
  CHECK(pr_apply_batch(g, ds, dd, nd, is, id, ni));
  pr_tuning tu;
  CHECK(pr_autotune(g, PR_DFP, 0.85, 1e-10, 1, &tu));
  pr_options host = {1e-6, 1e-6, 500, PR_OPT_HOST_LOOP};
  CHECK(pr_update(g, PR_DFP, 0.85, 1e-10, &host, &st));
  CHECK(pr_ranks(g, r1));
  const int32_t it_host = st.iterations;
  CHECK(pr_set_ranks(g, r0));
  pr_options dev = {1e-6, 1e-6, 500, PR_OPT_DEVICE_LOOP};
  CHECK(pr_update(g, PR_DFP, 0.85, 1e-10, &dev, &st));
  CHECK(pr_ranks(g, r2));
  pr_graph_destroy(g);
  FILE* f = fopen(argv[2], "wb");
  if (!f) return 4;
  fwrite(r0, sizeof(double), (size_t)n, f);
  fwrite(r1, sizeof(double), (size_t)n, f);
  fwrite(r2, sizeof(double), (size_t)n, f);
  fclose(f);
  printf("iterations host %d device %d tuned %d/%d/%d/%d\n", it_host, st.iterations, tu.threads, tu.quads_per_lane,
         tu.hub_vertices, tu.fused_epilogue);
  return 0;
}
"""


def test_c_program_runs_dfp_through_the_abi(tmp_path):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not found")
    from paper_2401_15870_gb300 import build
    lib = build.build()
    n = 1 << 13
    src, dst = synth.rmat(13, 16 * n, 777)
    order = np.lexsort((dst, src))
    s, d = src[order].astype(np.int32), dst[order].astype(np.int32)
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, s.astype(np.int64) + 1, 1)
    off = np.cumsum(off)
    O = oracle.Graph(n, s, d)
    cs, cd = synth.unique_edges(s, d)
    ds, dd, is_, id_ = synth.batch(n, cs, cd, 200, 778)
    np.array([n], np.int32).tofile(tmp_path / "n.bin")
    off.tofile(tmp_path / "off.bin")
    d.tofile(tmp_path / "col.bin")
    np.concatenate([[len(ds), len(is_)], ds, dd, is_, id_]).astype(np.int32).tofile(tmp_path / "batch.bin")
    (tmp_path / "main.c").write_text(PROGRAM)
    exe = tmp_path / "dfpr_c"
    libdir = os.path.dirname(lib)
    subprocess.check_call([gcc, "-O1", "-std=c11", "-I", os.path.join(ROOT, "include"), str(tmp_path / "main.c"),
                           "-L", libdir, "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir, "-o", str(exe)])
    out = tmp_path / "ranks.bin"
    r = subprocess.run([str(exe), str(tmp_path), str(out)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    ranks = np.fromfile(out, np.float64).reshape(3, n)
    ref0, _ = O.update("static")
    assert np.max(np.abs(ranks[0] - ref0)) < TOL
    O.apply_batch(ds, dd, is_, id_)
    ref, _ = O.update("dfp", r_prev=ranks[0])
    assert np.max(np.abs(ranks[1] - ref)) < TOL
    assert np.array_equal(ranks[1], ranks[2])
