"""The D3Q27h reconstruction of the fused kernel (`full_populations` in csrc/stream_collide.cuh,
the factorised complete-basis sum) compiled for the host with g++ and compared with the oracle's
full-basis sum on random moments, forces and relaxation rates. The GPU parity tests check the whole
step; this checks the arithmetic of the staging on a machine without a GPU."""
import os
import shutil
import subprocess

import pytest
import torch

import oracle
from oracle import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2609_09160_gb300", "csrc", "stream_collide.cuh")

HARNESS = r'''
#include <cstdio>
%s
int main() {
  int n;
  if (scanf("%%d", &n) != 1) return 1;
  for (int t = 0; t < n; ++t) {
    double p, u[3], h[3], N6[6], omm;
    if (scanf("%%lf %%lf %%lf %%lf %%lf %%lf %%lf %%lf %%lf %%lf %%lf %%lf %%lf %%lf", &p, &u[0], &u[1], &u[2],
              &h[0], &h[1], &h[2], &N6[0], &N6[1], &N6[2], &N6[3], &N6[4], &N6[5], &omm) != 14)
      return 1;
    const double Nt[3][3] = {{N6[0], N6[3], N6[4]}, {N6[3], N6[1], N6[5]}, {N6[4], N6[5], N6[2]}};
    double g[27];
    full_populations<double>(p, u, h, Nt, omm, g);
    for (int q = 0; q < 27; ++q) printf("%%.17g ", g[q]);
    printf("\n");
  }
  return 0;
}
'''


def _extract_function():
    src = open(HEADER).read()
    start = src.index("template <class T>\n__device__ __forceinline__ void full_populations")
    end = src.index("\n}\n", start) + 3
    return src[start:end].replace("__device__ __forceinline__", "inline")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_full_populations_matches_the_oracle(tmp_path):
    cpp = tmp_path / "full.cpp"
    exe = tmp_path / "full"
    cpp.write_text(HARNESS % _extract_function())
    subprocess.run(["g++", "-O1", "-std=c++17", "-o", str(exe), str(cpp)], check=True, capture_output=True)
    g = torch.Generator().manual_seed(11)
    cases, lines = [], []
    for _ in range(24):
        p = 1e-2 * torch.randn((), generator=g, dtype=torch.float64)
        u = 0.1 * torch.randn(3, generator=g, dtype=torch.float64)
        F = 1e-3 * torch.randn(3, generator=g, dtype=torch.float64)
        N = 1e-2 * torch.randn(3, 3, generator=g, dtype=torch.float64)
        N = 0.5 * (N + N.T)
        om = 1.0 + 0.9 * torch.rand((), generator=g, dtype=torch.float64)
        cases.append((p, u, N, F, om))
        h = F / 2  # rho = 1
        vals = [p, *u, *h, N[0, 0], N[1, 1], N[2, 2], N[0, 1], N[0, 2], N[1, 2], 1 - om]
        lines.append(" ".join(repr(float(v)) for v in vals))
    out = subprocess.run([str(exe)], input=f"{len(lines)}\n" + "\n".join(lines) + "\n", capture_output=True,
                         text=True, check=True).stdout.split("\n")
    lat = oracle.D3Q27H
    one = torch.ones(1, dtype=torch.float64)
    for (p, u, N, F, om), line in zip(cases, out):
        got = torch.tensor([float(x) for x in line.split()], dtype=torch.float64)
        coefs = lbm.full_coefficients(lat, p.reshape(1), u.reshape(3, 1), N.reshape(3, 3, 1), F.reshape(3, 1), one,
                                      om.reshape(1))
        want = lbm.full_reconstruct(lat, coefs)[:, 0] / lat.w  # kernel cube order = oracle order
        assert float((got - want).abs().max() / want.abs().max()) < 1e-14
