"""Planted mistakes: the oracle's pins must reject every plausible slip.

Each variant below carries one mistake of the kinds that slip into code like
the oracle's -- a wrong sign, a dropped term or factor, a transposed operand,
a wrong index, an inverted order -- planted in a patched copy of the oracle
sources in a temporary directory (the committed oracle is not touched). Every
variant is compiled on the CPU and the pin tests that cover its part of the
method are run against it; each variant must make at least one pin fail. A
variant that passed would mean that part of the oracle is not pinned.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")
PINS = "tests/test_oracle_pins.py"
ENV_PINS = "tests/test_oracle_envmap.py"
CONTRACT_PINS = "tests/test_oracle_contract.py"

# name: (source file, exact text, replacement, pin file)
MUTANTS = {
    # projection (Sec. 2 pinhole model) and footprints (Sec. 3.2)
    "rotation transposed": (
        "oracle.cpp", "T xc = R[0] * x; xc = xc + R[1] * y; xc = xc + R[2] * z;",
        "T xc = R[0] * x; xc = xc + R[3] * y; xc = xc + R[6] * z;", PINS),
    "principal point sign": (
        "oracle.cpp", "T qx = xc / zc; T u = fx * qx; u = u + cx;",
        "T qx = xc / zc; T u = fx * qx; u = u - cx;", PINS),
    "pixel centres at integers": (
        "oracle.cpp", "const T um = u - half, vm = v - half;", "const T um = u, vm = v;", PINS),
    "bilinear weights swapped": (
        "oracle.cpp", "const double wx64 = (px == sp.i0) ? 1.0 - sp.a : sp.a;",
        "const double wx64 = (px == sp.i0) ? sp.a : 1.0 - sp.a;", PINS),
    "bilinear fraction index": (
        "oracle.cpp", "const T a = um - fi, b = vm - fj;", "const T a = um - fi, b = um - fi;", PINS),
    "alpha not clamped": (
        "oracle.cpp",
        "fr.w_or_g = wx64 * wy64;\n        fr.alpha = fr.unclamped ? opac * fr.w_or_g : (double)o.alpha_max;",
        "fr.w_or_g = wx64 * wy64;\n        fr.alpha = opac * fr.w_or_g;", PINS),
    "Gaussian cross term halved": (
        "oracle.cpp", "const double m64 = sp.ca * dx64 * dx64 + 2.0 * sp.cb",
        "const double m64 = sp.ca * dx64 * dx64 + sp.cb", PINS),
    "dilation dropped on one axis": (
        "oracle.cpp", "S00 = s2 * d0; S00 = S00 + dil;", "S00 = s2 * d0;", PINS),
    "truncation at 2 sigma": ("oracle.cpp", "r = (T)3 * r;", "r = (T)2 * r;", PINS),
    "conic off-diagonal sign": ("oracle.cpp", "cb = -(S01 / det)", "cb = (S01 / det)", PINS),
    "Jacobian sign": ("oracle.cpp", "j02 = j02 / zz; j02 = -j02;", "j02 = j02 / zz;", PINS),
    "Gaussian value exp(-m)": (
        "oracle.cpp", "fr.w_or_g = std::exp(-0.5 * m64);", "fr.w_or_g = std::exp(-m64);", PINS),
    "coverage cut at 2 sigma": (
        "oracle.cpp", "if (!(m <= (T)9)) return false;", "if (!(m <= (T)4)) return false;", PINS),
    "default scale inverted": (
        "oracle.cpp", "T s = has_scale ? (T)scale : (T)((T)5 * nearT / fx);",
        "T s = has_scale ? (T)scale : (T)((T)5 * fx / nearT);", PINS),
    "isotropic covariance over z": (
        "oracle.cpp", "T ff = fx * fy; ff = ff / zz;", "T ff = fx * fy; ff = ff / zc;", PINS),
    # sorting (Sec. 2 depth-sorted lists; Sec. 3.2 tile lists)
    "pixel lists back to front": (
        "oracle.cpp",
        "std::stable_sort(pts.begin() + start[k], pts.begin() + start[k + 1],\n"
        "                         [&](int32_t p, int32_t q) { return c.sp[p].zbits < c.sp[q].zbits; });",
        "std::stable_sort(pts.begin() + start[k], pts.begin() + start[k + 1],\n"
        "                         [&](int32_t p, int32_t q) { return c.sp[p].zbits > c.sp[q].zbits; });",
        PINS),
    "tile lists back to front": (
        "oracle.cpp",
        "std::stable_sort(tl.pts.begin() + tl.start[t], tl.pts.begin() + tl.start[t + 1],\n"
        "                         [&](int32_t p, int32_t q) { return c.sp[p].zbits < c.sp[q].zbits; });",
        "std::stable_sort(tl.pts.begin() + tl.start[t], tl.pts.begin() + tl.start[t + 1],\n"
        "                         [&](int32_t p, int32_t q) { return c.sp[p].zbits > c.sp[q].zbits; });",
        PINS),
    # compositing (Eq. 1)
    "transmittance never falls": ("oracle.cpp", "T64 *= (1.0 - fr.alpha);", "T64 *= 1.0;", PINS),
    "termination tested before the step": (
        "oracle.cpp", "if (nxt < tmin) {", "if (Tdec < tmin) {", PINS),
    "transmittance dropped from the weight": (
        "oracle.cpp", "const double w = T64 * fr.alpha;", "const double w = fr.alpha;", PINS),
    "depth not weighted": ("oracle.cpp", "D += w * c.sp[i].zc;", "D += fr.alpha * c.sp[i].zc;", PINS),
    # adjoint (appendix, corrected Eq. 2)
    "background term sign": ("oracle.cpp", "da += gA * Tfin / om;", "da -= gA * Tfin / om;", PINS),
    "replay divisor sign": (
        "oracle.cpp", "const double a = b.fr.alpha, Tk = b.T, om = 1.0 - a;",
        "const double a = b.fr.alpha, Tk = b.T, om = 1.0 + a;", PINS),
    "depth term dropped": (
        "oracle.cpp", "da += gD * (Tk * c.sp[b.pt].zc - SD / om);", "da += gD * (Tk * c.sp[b.pt].zc);", PINS),
    "suffix sum without T": ("oracle.cpp", "S[j] += a * Tk * f[j];", "S[j] += a * f[j];", PINS),
    "feature gradient without alpha": (
        "oracle.cpp", "dfs[q * C + j] = Tk * a * gF[j];", "dfs[q * C + j] = Tk * gF[j];", PINS),
    "opacity gradient without weight": (
        "oracle.cpp", "d_opacity[i] += e.fr.w_or_g * e.dalpha;", "d_opacity[i] += e.dalpha;", PINS),
    "gradient through the alpha clamp": (
        "oracle.cpp", "if (!e.fr.unclamped) continue;", "(void)0;", PINS),
    "screen gradient conic index": (
        "oracle.cpp", "du[i] += dm * -(2.0 * s.ca * e.fr.dx + 2.0 * s.cb * e.fr.dy);",
        "du[i] += dm * -(2.0 * s.ca * e.fr.dx + 2.0 * s.cc * e.fr.dy);", PINS),
    "depth chain sign": (
        "oracle.cpp", "gz += du[i] * (-fx * x / (z * z))", "gz += du[i] * (fx * x / (z * z))", PINS),
    "world gradient not transposed": (
        "oracle.cpp", "d_xyz[3 * i + 0] = R[0] * gx + R[3] * gy + R[6] * gz;",
        "d_xyz[3 * i + 0] = R[0] * gx + R[1] * gy + R[2] * gz;", PINS),
    "isotropic scale gradient factor": (
        "oracle.cpp", "gs += dS * 2.0 * sc * fx * fy / z2;", "gs += dS * sc * fx * fy / z2;", PINS),
    # background model (Sec. 3.2 "Faster Background Model Evaluation")
    "map direction not rotated back": (
        "envmap.cpp",
        "dw[i] = (double)c.R[0 * 3 + i] * dc[0] + (double)c.R[1 * 3 + i] * dc[1] + (double)c.R[2 * 3 + i] * dc[2];",
        "dw[i] = (double)c.R[i * 3 + 0] * dc[0] + (double)c.R[i * 3 + 1] * dc[1] + (double)c.R[i * 3 + 2] * dc[2];",
        ENV_PINS),
    "longitude axes swapped": ("envmap.cpp", "std::atan2(dw[0], dw[2])", "std::atan2(dw[2], dw[0])", ENV_PINS),
    "texel rows not centred": (
        "envmap.cpp", "const double Y = th / pi * Hb - 0.5;", "const double Y = th / pi * Hb;", ENV_PINS),
    "longitude clamped, not wrapped": (
        "envmap.cpp", "v %= Wb; return v < 0 ? v + Wb : v;", "return v < 0 ? 0 : (v > Wb - 1 ? Wb - 1 : v);",
        ENV_PINS),
    "background alpha gradient sign": ("envmap.cpp", "da -= g[p * C + c] * v;", "da += g[p * C + c] * v;", ENV_PINS),
    "map gradient ignores coverage": (
        "envmap.cpp", "+= t.w[k] * (1.0 - alpha[p]) * g[p * C + c];", "+= t.w[k] * g[p * C + c];", ENV_PINS),
    # spherical contraction (Sec. 3.4)
    "contraction not normalised": ("envmap.cpp", "(2.0 - 1.0 / r) / r", "(2.0 - 1.0 / r)", CONTRACT_PINS),
}


def _run_variant(name, tmp):
    src_name, old, new, pins = MUTANTS[name]
    d = os.path.join(tmp, "".join(ch if ch.isalnum() else "_" for ch in name))
    os.makedirs(d)
    srcs = []
    for f in ("oracle.cpp", "envmap.cpp"):
        text = open(os.path.join(ORACLE_DIR, f)).read()
        if f == src_name:
            assert text.count(old) == 1, f"{name}: the planted text must occur once in {f}"
            text = text.replace(old, new)
        path = os.path.join(d, f)
        with open(path, "w") as fh:
            fh.write(text)
        srcs.append(path)
    lib = os.path.join(d, "liboracle.so")
    subprocess.run(oracle.compile_command(srcs, lib), check=True, capture_output=True)
    env = dict(os.environ, INPC_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", pins, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    return name, r.returncode, r.stdout[-600:]


def test_every_planted_mistake_fails_a_pin():
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            results = list(ex.map(lambda n: _run_variant(n, tmp), MUTANTS))
    survived = [(n, out) for n, rc, out in results if rc == 0]
    broken = [(n, rc, out) for n, rc, out in results if rc not in (0, 1)]
    assert not broken, broken  # 1 = some pin failed; anything else is a harness error
    assert not survived, "mistakes no pin catches: " + ", ".join(n for n, _ in survived)
