"""A plain C program against the C ABI (no Python, no PyTorch): it describes a
one-patch unit cube (p = 1, 2^3 elements, identity map, half of it conducting),
creates a host-only context (device -1: setup, gauge and queries, no GPU), reads the
DOF count and the gauge classes, assembles a coil load vector, checks a rejected
option's error code and message, and destroys the context.  Built with the host
compiler against libieti.so; the numbers it prints are checked against the same
queries through the Python binding."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "ieti.h"

int main(void) {
  const int ne = 2, p = 1;                   /* elements, degree per direction */
  int32_t n_el[1] = {ne}, deg[1] = {p};
  double knots[5] = {0, 0, 0.5, 1, 1};       /* open knot vector of 2 elements, degree 1 */
  const int n = ne + p;                      /* control points per direction */
  double ctrl[27 * 3];
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        double *c = ctrl + 3 * (i + n * (j + n * k));
        c[0] = 0.5 * i; c[1] = 0.5 * j; c[2] = 0.5 * k;   /* knot averages: identity map */
      }
  double sigma[8], nu[8];
  for (int e = 0; e < 8; ++e) { sigma[e] = (e % 2 == 0) ? 1.0 : 0.0; nu[e] = 1.0; }
  ieti_problem pr;
  memset(&pr, 0, sizeof pr);
  for (int d = 0; d < 3; ++d) { pr.n_patches[d] = 1; pr.n_el[d] = n_el; pr.degree[d] = deg; pr.knots[d] = knots; }
  pr.ctrl_pts = ctrl; pr.sigma_el = sigma; pr.nu_el = nu; pr.dt = 0.01;
  ieti_options op;
  memset(&op, 0, sizeof op);
  op.device = -1; op.precision = IETI_PREC_FP64; op.precond = IETI_PRECOND_DIRICHLET;
  op.cg_tol = 1e-10; op.cg_max_it = 100; op.max_sweeps = 1;
  ieti_ctx *ctx = NULL;
  int rc = ieti_setup(&pr, &op, &ctx);
  if (rc != 0) { printf("setup %d %s\n", rc, ieti_setup_error()); return 1; }
  int64_t N = ieti_num_dofs(ctx);
  int8_t *cls = malloc(N), *tree = malloc(N);
  double *j = malloc(N * sizeof(double));
  rc = ieti_dof_classes(ctx, cls, tree);
  int counts[3] = {0, 0, 0};
  for (int64_t k = 0; k < N; ++k) counts[cls[k]]++;
  ieti_coil coil = {1.0, 0.3, 0.45, 0.5, 0.5, 0.5, 0.2};
  rc |= ieti_load_vector(ctx, &coil, j);
  double s = 0;
  for (int64_t k = 0; k < N; ++k) s += j[k] * j[k];
  printf("dofs %lld classes %d %d %d loadnorm2 %.17g rc %d\n", (long long)N, counts[0], counts[1], counts[2], s, rc);
  op.cg_tol = 2.0;                           /* outside (0, 1): refused */
  ieti_ctx *bad = NULL;
  rc = ieti_setup(&pr, &op, &bad);
  printf("bad %d %s\n", rc, ieti_setup_error());
  ieti_destroy(ctx);
  free(cls); free(tree); free(j);
  return 0;
}
"""


def test_plain_c_client():
    cc = shutil.which("cc") or shutil.which("gcc")
    if not cc:
        pytest.skip("no C compiler")
    from paper_2510_23446_gb300.build import build
    build()
    from paper_2510_23446_gb300 import ieti
    libdir = os.path.dirname(ieti.LIB_PATH)
    with tempfile.TemporaryDirectory() as tmp:
        src, exe = os.path.join(tmp, "client.c"), os.path.join(tmp, "client")
        open(src, "w").write(C_SRC)
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe, "-L", libdir, "-lieti",
                        f"-Wl,-rpath,{libdir}"], check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    lines = out.stdout.strip().splitlines()
    f = lines[0].split()
    n_dofs, c0, c1, c2, norm2 = int(f[1]), int(f[3]), int(f[4]), int(f[5]), float(f[7])
    assert int(f[9]) == 0
    assert n_dofs == 3 * 2 * 3 * 3 and c0 + c1 + c2 == n_dofs     # 3 directions x 2 x 3 x 3 edges
    assert c0 > 0                                                  # boundary edges eliminated
    bad = lines[1].split(maxsplit=2)
    assert int(bad[1]) == -1 and "cg_tol" in bad[2]
    # the same queries through the binding on the same description
    S = ieti.Solver([1, 1, 1], [[2]] * 3, [[1]] * 3, [np.array([0, 0, 0.5, 1, 1.0])] * 3,
                    _ctrl(), np.array([1.0, 0.0] * 4), np.ones(8), 0.01, device=-1, precond="dirichlet")
    cls, _ = S.dof_classes()
    j = S.load_vector(dict(J0=1.0, r_in=0.3, r_out=0.45, xc=0.5, yc=0.5, zc=0.5, hz=0.2))
    assert S.n == n_dofs and [int(np.sum(cls == c)) for c in range(3)] == [c0, c1, c2]
    assert abs(float(j @ j) - norm2) <= 1e-12 * max(norm2, 1e-300)
    S.close()


def _ctrl():
    n = 3
    c = np.zeros((n, n, n, 3))
    for k in range(n):
        for jj in range(n):
            for i in range(n):
                c[k, jj, i] = (0.5 * i, 0.5 * jj, 0.5 * k)
    return c.ravel()
