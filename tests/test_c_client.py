"""A plain C program uses the library through include/soma.h alone: no Python
and no PyTorch on its side.  On CPU it compiles, links against libsoma.so
and meets the missing device with a CUDA error code; on a GPU it creates a
system, steps it and reads counts and observables back."""
import os
import subprocess
import tempfile

import pytest

from paper_2606_09356_b300 import build as _build
from paper_2606_09356_b300 import soma

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "soma.h"

int main(void) {
  soma_system_desc d;
  memset(&d, 0, sizeof d);
  d.n_poly = 512; d.N = 32; d.n_A = 16;
  d.grid[0] = d.grid[1] = d.grid[2] = 16;
  d.box[0] = d.box[1] = d.box[2] = 4.0;
  d.chiN = 20.0; d.kappaN = 50.0; d.seed = 1; d.move = SOMA_MOVE_UNIFORM;
  soma_options o;
  soma_options_default(&o);
  soma_handle* h = NULL;
  int rc = soma_create(&d, 1, &o, &h);
  if (rc != SOMA_OK) {
    printf("create %d %s\n", rc, soma_strerror(rc));
    return 2;
  }
  if ((rc = soma_mc_steps(h, 10, NULL)) != SOMA_OK) { printf("steps %d\n", rc); return 3; }
  const size_t nc = 16 * 16 * 16;
  uint32_t* counts = (uint32_t*)malloc(sizeof(uint32_t) * 2 * nc);
  if ((rc = soma_get_density(h, 0, counts, 2 * nc, SOMA_HOST)) != SOMA_OK) { printf("density %d\n", rc); return 4; }
  unsigned long long a = 0, b = 0;
  for (size_t c = 0; c < nc; ++c) { a += counts[c]; b += counts[nc + c]; }
  soma_obs obs;
  if ((rc = soma_observables(h, 0, &obs)) != SOMA_OK) { printf("observables %d\n", rc); return 5; }
  printf("ok %llu %llu %llu %.4f\n", a, b, (unsigned long long)obs.step, obs.acc);
  free(counts);
  soma_destroy(h);
  return 0;
}
'''


def _compile(td):
    _build.build()
    c = os.path.join(td, "client.c")
    exe = os.path.join(td, "client")
    open(c, "w").write(SRC)
    libdir = os.path.dirname(soma.LIBRARY)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-o", exe, c,
                           "-L", libdir, "-lsoma", "-Wl,-rpath," + libdir])
    return exe


def test_c_client_builds_and_reports_missing_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the GPU test runs the client")
    with tempfile.TemporaryDirectory() as td:
        out = subprocess.run([_compile(td)], capture_output=True, text=True)
    assert out.returncode == 2, out.stdout + out.stderr
    assert out.stdout.startswith(f"create {soma.SOMA_ECUDA} ")


@pytest.mark.gpu
def test_c_client_runs():
    with tempfile.TemporaryDirectory() as td:
        out = subprocess.run([_compile(td)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    tag, a, b, step, acc = out.stdout.split()
    assert tag == "ok" and int(a) == 512 * 16 and int(b) == 512 * 16 and int(step) == 10
    assert 0.3 < float(acc) < 0.9
