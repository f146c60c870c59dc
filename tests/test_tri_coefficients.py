"""The TRI kernels' spin coefficients (`csrc/tri_coef.h`, hand-derived Pauli phases evaluated at
compile time) against the oracle's literal Pauli contraction (no GPU).

The header is compiled on the host with g++ into a small dump program; its dense tables, in the
kernels' real storage (Gamma^{mu nu} = i g^{mu nu} for the six imaginary-class functions), must
equal the oracle's complex tables converted to that storage, for the five terms of the vertex
flow and the exchange part of the correlation.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(os.path.dirname(HERE), "paper_2109_13317_gb300", "csrc", "tri_coef.h")

DUMP = r"""
#define __host__
#define __device__
#include "tri_coef.h"
#include <cstdio>
using namespace sr::tri;
int main() {
  for (int mu = 0; mu < 4; ++mu) for (int nu = 0; nu < 4; ++nu) {
    const int o = mu * 4 + nu;
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) {
      std::printf("0 %d %d %d %d\n", o, a * 4 + b, (a ^ mu) * 4 + (b ^ nu), coef_s(mu, nu, a, b));
      std::printf("4 %d %d %d %d\n", o, a * 4 + b, (a ^ mu) * 4 + (b ^ nu), coef_u(mu, nu, a, b));
    }
    for (int l = 0; l < 4; ++l) std::printf("1 %d %d %d %d\n", o, mu * 4 + l, l * 4 + nu, 2 * coef_t(mu, nu, l));
    for (int l = 0; l < 4; ++l) for (int m = 0; m < 4; ++m) {
      std::printf("2 %d %d %d %d\n", o, mu * 4 + l, m * 4 + (m ^ l ^ nu), coef_o2(mu, nu, l, m));
      std::printf("3 %d %d %d %d\n", o, (mu ^ l ^ m) * 4 + l, m * 4 + nu, coef_o3(mu, nu, l, m));
    }
    for (int l = 0; l < 4; ++l) std::printf("9 %d %d 0 %d\n", o, (mu ^ nu ^ l) * 4 + l, 2 * coef_x(mu, nu, l));
  }
  return 0;
}
"""


def _iota(c):
    return 1 if ((c // 4) == 0) != ((c % 4) == 0) else 0


def test_kernel_coefficients_equal_oracle_contraction(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "dump.cpp"
    src.write_text(DUMP)
    exe = tmp_path / "dump"
    subprocess.check_call([gxx, "-std=c++17", "-O0", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True)
    G = np.zeros((5, 16, 16, 16))
    GX = np.zeros((16, 16))
    for line in out.splitlines():
        t, o, x, y, c = map(int, line.split())
        if t == 9:
            GX[o, x] += c
        else:
            G[t, o, x, y] += c
    coef, _, _, _, cexc = O.tri_spin_tables()
    R = np.zeros((5, 16, 16, 16))
    for t in range(5):
        for o in range(16):
            for x in range(16):
                for y in range(16):
                    v = coef[t, o, x, y] * (1j) ** (_iota(x) + _iota(y) - _iota(o))
                    assert abs(v.imag) < 1e-12
                    R[t, o, x, y] = v.real
    X = np.zeros((16, 16))
    for o in range(16):
        for x in range(16):
            v = cexc[o, x] * (1j) ** (_iota(x) - _iota(o))
            assert abs(v.imag) < 1e-12
            X[o, x] = v.real
    for t in range(5):
        np.testing.assert_array_equal(G[t], R[t], err_msg=f"term {t}")
        assert np.count_nonzero(R[t]) == (64 if t == 1 else 256)
    np.testing.assert_array_equal(GX, X)
