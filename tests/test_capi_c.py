"""The C ABI used from plain C: a C99 program includes include/pufe.h, links
libpufe.so, builds a small cell's mesh, reads its sizes and CSR pattern, and
exercises the error paths.  Its sizes must equal those the Python binding
reports for the same cell.  Needs no GPU (without one, compute calls report
PUFE_ESTATE)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1611_00731_gb300 import pufe
from paper_1611_00731_gb300.build import LIBDIR

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "pufe.h"

int main(void) {
  /* H-like atom at the origin, Li-like atom at the cell centre */
  const double tau[6] = {0.0, 0.0, 0.0, 2.0, 2.0, 2.0};
  const int spec[2] = {0, 1};
  const int n0[1] = {1}, l0[1] = {0}, m0[1] = {0};
  const double z0[1] = {1.0};
  const int n1[5] = {1, 2, 2, 2, 2}, l1[5] = {0, 0, 1, 1, 1}, m1[5] = {0, 0, -1, 0, 1};
  const double z1[5] = {2.70, 0.65, 0.65, 0.65, 0.65};
  pufe_species sp[2] = {{1, n0, l0, m0, z0, 1.5, 1.5}, {5, n1, l1, m1, z1, 1.5, 1.5}};
  pufe_cell cell = {{4.0, 4.0, 4.0}, {2, 2, 2}, 2, tau, spec, NULL, PUFE_FE_LAGRANGE64};
  pufe_quad quad = {PUFE_QUAD_FIXED, 4, 4, 0, 0, 1e-6, 0, 0};
  pufe_ctx *ctx = NULL;
  pufe_status s;
  int64_t N = 0, nnz = 0, nq = 0, ne = 0, nb = 0, i;
  int64_t *rowptr;
  int32_t *col;

  /* an invalid cell is rejected with a message and no context */
  cell.nel[1] = 0;
  s = pufe_build_mesh(&cell, sp, 2, &quad, &ctx);
  if (s != PUFE_EINVAL || ctx != NULL || pufe_last_error()[0] == '\0') return 10;
  cell.nel[1] = 2;

  s = pufe_build_mesh(&cell, sp, 2, &quad, &ctx);
  if (s != PUFE_OK || ctx == NULL) return 11;
  if (pufe_get_sizes(ctx, &N, &nnz, &nq, &ne, &nb) != PUFE_OK) return 12;
  rowptr = (int64_t *)malloc((size_t)(N + 1) * sizeof(int64_t));
  col = (int32_t *)malloc((size_t)nnz * sizeof(int32_t));
  if (!rowptr || !col) return 13;
  if (pufe_get_pattern(ctx, rowptr, col) != PUFE_OK) return 14;
  if (rowptr[0] != 0 || rowptr[N] != nnz) return 15;
  for (i = 0; i < N; ++i) {
    int64_t j;
    if (rowptr[i + 1] <= rowptr[i]) return 16;            /* every row has its diagonal */
    for (j = rowptr[i] + 1; j < rowptr[i + 1]; ++j)
      if (col[j] <= col[j - 1] || col[j] >= N) return 17;  /* sorted, in range */
  }
  s = pufe_tabulate(ctx, PUFE_FP64, NULL);
  if (s != PUFE_OK && s != PUFE_ESTATE) return 18;
  if (s == PUFE_ESTATE && pufe_last_error()[0] == '\0') return 19;
  printf("%lld %lld %lld %lld %lld\n", (long long)N, (long long)nnz, (long long)nq,
         (long long)ne, (long long)nb);
  free(rowptr);
  free(col);
  pufe_destroy(ctx);
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_c_program_builds_a_mesh_through_the_header(tmp_path):
    pufe.load_library()
    src = tmp_path / "prog.c"
    exe = tmp_path / "prog"
    src.write_text(PROGRAM)
    cc = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
          "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
          "-L", LIBDIR, "-lpufe", f"-Wl,-rpath,{LIBDIR}"]
    r = subprocess.run(cc, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    N, nnz, nq, ne, nb = (int(v) for v in r.stdout.split())

    from paper_1611_00731_gb300 import workloads as W
    ctx = pufe.pufe_build_mesh(W.small_two_atom(nel=2, a=4.0, quad_p=4))
    n_e, _ = ctx.element_basis()
    assert (N, nnz, nq, ne, nb) == (ctx.n_dof, ctx.nnz, ctx.n_q, ctx.n_elem,
                                    int(np.max(n_e)))
