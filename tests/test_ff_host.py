"""The float-float arithmetic of the setup pass (osog_ff.h), compiled for the
host and checked against numpy's float64 math: cos and sin of float angles
(Cody-Waite reduction and Taylor series), reciprocals, and the ellipse row
quadric m, 1/alpha, kappa, sqrt(alpha) that the raster evaluates near the
rim.  The header is the device code itself: on the GPU its operations are
the same IEEE float operations with rounding to nearest (the _rn
intrinsics), here plain float operations built without contraction."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(__file__), os.pardir, "paper_2606_21381_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "osog_ff.h"
using namespace osog;
// stdin: n, then n records (th, a, b) as float bits; stdout: per record the
// float bits of cos, sin, 1/a (h, l each) and of m, 1/alpha, kappa,
// sqrt(alpha) (h, l each)
int main() {
    int n = 0;
    if (std::fread(&n, sizeof n, 1, stdin) != 1) return 1;
    std::vector<float> in(3 * (size_t)n);
    if (std::fread(in.data(), sizeof(float), in.size(), stdin) != in.size()) return 1;
    std::vector<float> out;
    for (int i = 0; i < n; ++i) {
        const float th = in[3 * i], a = in[3 * i + 1], b = in[3 * i + 2];
        ff c, s;
        ff_sincos(th, &c, &s);
        const ff ia = ff_recip(a);
        const Quadric q = ellipse_quadric(a, b, c, s);
        const ff v[7] = {c, s, ia, q.m, q.inv_alpha, q.kappa, q.sqrt_alpha};
        for (const ff &x : v) {
            out.push_back(x.h);
            out.push_back(x.l);
        }
    }
    std::fwrite(out.data(), sizeof(float), out.size(), stdout);
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("ff")
    src, exe = d / "ff.cpp", d / "ff"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC, str(src), "-o",
                    str(exe)], check=True)
    return exe


def run(exe, th, a, b):
    th, a, b = (np.asarray(v, np.float32) for v in (th, a, b))
    rec = np.stack([th, a, b], axis=1).astype(np.float32)
    payload = np.int32(len(rec)).tobytes() + rec.tobytes()
    res = subprocess.run([str(exe)], input=payload, capture_output=True, check=True)
    v = np.frombuffer(res.stdout, np.float32).reshape(len(rec), 7, 2).astype(np.float64)
    return v[..., 0] + v[..., 1], v


def angles():
    rng = np.random.default_rng(0)
    quarter = np.float32(math.pi / 4)
    edges = np.array([np.nextafter(np.float32(k) * quarter, np.float32(s * np.inf))
                      for k in range(-16, 17) for s in (-1, 1)], np.float32)
    return np.concatenate([
        rng.uniform(-math.pi, math.pi, 20000), rng.uniform(-60.0, 60.0, 4000),
        rng.uniform(-2.0 ** 20, 2.0 ** 20, 2000), edges,
        [0.0, -0.0, 1e-30, -1e-20, 1e-8, 3e-4, 2.0 ** 20, -(2.0 ** 20)],
    ]).astype(np.float32)


def test_cos_sin_of_float_angles_to_2_pow_minus_46(harness):
    th = angles()
    got, parts = run(harness, th, np.ones_like(th), np.ones_like(th))
    t = th.astype(np.float64)
    err_c = np.abs(got[:, 0] - np.cos(t))
    err_s = np.abs(got[:, 1] - np.sin(t))
    assert err_c.max() <= 2.0 ** -46 and err_s.max() <= 2.0 ** -46, (err_c.max(), err_s.max())
    # normalised pairs: |l| <= ulp(h) / 2
    for k in (0, 1):
        h, l = parts[:, k, 0], parts[:, k, 1]
        assert np.all(np.abs(l) <= 0.5 * np.spacing(np.abs(h).astype(np.float32)).astype(np.float64))
    # exact special values
    z = np.nonzero(th == 0)[0]
    assert np.all(got[z, 0] == 1.0) and np.all(got[z, 1] == 0.0)
    # a tiny angle keeps its relative precision in sin
    tiny = np.nonzero((np.abs(t) > 0) & (np.abs(t) < 1e-6))[0]
    assert np.all(np.abs(got[tiny, 1] - np.sin(t[tiny])) <= 2.0 ** -46 * np.abs(t[tiny]))


def test_reciprocal_of_a_float_to_2_pow_minus_47(harness):
    rng = np.random.default_rng(1)
    a = np.concatenate([rng.uniform(0.3, 400.0, 5000), 2.0 ** rng.uniform(-20, 20, 2000),
                        [1.0, 3.0, 0.1, 7.0]]).astype(np.float32)
    got, _ = run(harness, np.zeros_like(a), a, np.ones_like(a))
    want = 1.0 / a.astype(np.float64)
    assert np.max(np.abs(got[:, 2] - want) / want) <= 2.0 ** -47


def test_ellipse_row_quadric_against_float64(harness):
    """m, 1/alpha, kappa and sqrt(alpha) of the semi-axes a, b (px) and the
    angle, against the definitions alpha = c^2/a^2 + s^2/b^2,
    m = -c s (1/a^2 - 1/b^2)/alpha, kappa = 1/(a^2 b^2 alpha^2) in float64:
    relative error below 2^-43 (m against its scale (b^2 - a^2)/(a^2 + b^2),
    since c s vanishes at the axes).  The float64 m is taken in the equal
    form -c s (b^2 - a^2) / (b^2 c^2 + a^2 s^2): with a close to b,
    1/a^2 - 1/b^2 cancels in float64 to about 1e-12 relative, while
    b^2 - a^2 of the exactly squared floats does not."""
    rng = np.random.default_rng(2)
    n = 20000
    th = np.concatenate([rng.uniform(-math.pi, math.pi, n), [0.0, math.pi / 2, 1e-7]])
    a = np.concatenate([rng.uniform(0.5, 300.0, n), [3.0, 3.0, 40.0]]).astype(np.float32)
    b = np.concatenate([a[:n] * rng.uniform(0.2, 5.0, n), [5.0, 5.0, 40.0]]).astype(np.float32)
    th = th.astype(np.float32)
    got, _ = run(harness, th, a, b)
    t, A, B = th.astype(np.float64), a.astype(np.float64), b.astype(np.float64)
    c, s = np.cos(t), np.sin(t)
    alpha = c * c / A ** 2 + s * s / B ** 2
    m = -c * s * (B ** 2 - A ** 2) / (B ** 2 * c * c + A ** 2 * s * s)
    inv_alpha = 1 / alpha
    kappa = 1 / (A ** 2 * B ** 2 * alpha ** 2)
    scale_m = np.abs(B ** 2 - A ** 2) / (A ** 2 + B ** 2) + 1e-300
    assert np.max(np.abs(got[:, 3] - m) / np.maximum(np.abs(m), scale_m)) <= 2.0 ** -43
    for k, want in ((4, inv_alpha), (5, kappa), (6, np.sqrt(alpha))):
        assert np.max(np.abs(got[:, k] - want) / want) <= 2.0 ** -43, k
    # a circle: m = 0 and 1/alpha = a^2 at every angle
    circ = np.nonzero(A == B)[0]
    assert np.all(got[circ, 3] == 0.0)
    assert np.max(np.abs(got[circ, 4] - A[circ] ** 2) / A[circ] ** 2) <= 2.0 ** -46
