"""Planted mistakes: each plausible slip in the oracle must fail a pin.

Every case copies the oracle into a scratch directory, plants one mistake
(a flipped sign, a dropped term, a transposed operand, a wrong index, an off
by one), and runs the pins of test_oracle_pins.py against the copy on the
CPU.  A mistake the pins do not notice fails this test.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_MUTATIONS = [
    ("fill rule, vertical sense", "return dy < 0 || (dy == 0 && dx < 0);",
     "return dy > 0 || (dy == 0 && dx < 0);"),
    ("fill rule, horizontal sense", "return dy < 0 || (dy == 0 && dx < 0);",
     "return dy < 0 || (dy == 0 && dx > 0);"),
    ("sample off the pixel centre", "int64_t px = 256 * x + 128, py = 256 * y + 128;",
     "int64_t px = 256 * x + 128, py = 256 * y;"),
    ("depth, wrong iz index", "float s2 = (float)E2 * iz[2];", "float s2 = (float)E2 * iz[1];"),
    ("depth, dropped term", "            s = s + s2;\n", "            s = s + 0.0f * s2;\n"),
    ("word, 4 mantissa bits dropped", "memcpy(&bits, &depth, 4);\n            uint64_t key = ((uint64_t)(bits >> 3) << 36)",
     "memcpy(&bits, &depth, 4);\n            uint64_t key = ((uint64_t)(bits >> 4) << 36)"),
    ("transform, dropped translation", "        s = s + mv[4 * r + 3];\n", "        s = s + 0.0f;\n"),
    ("transform, dropped z term", "        s = s + c;\n        s = s + mv", "        s = s + 0.0f * c;\n        s = s + mv"),
    ("model-view, transposed product", "(double)view[4 * r + k] * (double)model[4 * k + c]",
     "(double)model[4 * r + k] * (double)view[4 * k + c]"),
    ("camera, fx and fy swapped", "float fx = proj[0], fy = proj[5]", "float fx = proj[5], fy = proj[0]"),
    ("clip, t from the outside value", "    float t = fin / den;", "    float t = fout / den;"),
    ("clip, left guard sign", "return v.x + ORC_GUARD * v.w;", "return v.x - ORC_GUARD * v.w;"),
    ("snap, truncation", "*X = (int32_t)rintf(xs);", "*X = (int32_t)xs;"),
    ("snap, ties away from zero", "*Y = (int32_t)rintf(ys);", "*Y = (int32_t)roundf(ys);"),
    ("screen, y down", "float py = sy + 1.0f;", "float py = 1.0f - sy;"),
    ("edge function reversed", "int64_t E1 = edge(X[2], Y[2], X[0], Y[0], px, py);",
     "int64_t E1 = edge(X[0], Y[0], X[2], Y[2], px, py);"),
    ("bbox clamp off by one", "if (x1 > W - 1) x1 = W - 1;", "if (x1 > W - 2) x1 = W - 2;"),
    ("no backface cull", "        if (cull_back) return;\n", "        if (0) return;\n"),
    ("id bases off by one", "        base[i] = acc;\n", "        base[i] = acc + (i > 0);\n"),
    ("resolve, lower bound", "if (a[mid] <= key) lo = mid + 1;", "if (a[mid] < key) lo = mid + 1;"),
    ("resolve, sign of w", "qv);\n    float w = dot3(r, qv) / det;", "qv);\n    float w = -dot3(r, qv) / det;"),
    ("resolve, ray fx and fy swapped", "float r[3] = {ndx / cp[0], ndy / cp[1], -1.0f};",
     "float r[3] = {ndx / cp[1], ndy / cp[0], -1.0f};"),
    ("resolve, pixel centre", "float ndx = ((float)(2 * x + 1) / (float)cam->W) - 1.0f;",
     "float ndx = ((float)(2 * x) / (float)cam->W) - 1.0f;"),
    ("interpolation, wrong colour index", "    float q = b[1] * c1;", "    float q = b[1] * c2;"),
    ("resolve, upper clamp of RGBA8 dropped",
     "            float c = out[ch];\n            if (!(c >= 0.0f)) c = 0.0f;\n            if (c > 1.0f) c = 1.0f;",
     "            float c = out[ch];\n            if (!(c >= 0.0f)) c = 0.0f;"),
    ("box filter, divides by ss", "    const float n = (float)(ss * ss);", "    const float n = (float)(ss);"),
    ("box filter, wrong sample row", "size_t f = (size_t)(ss * y + sy) * (size_t)Wf", "size_t f = (size_t)(ss * y + sx) * (size_t)Wf"),
    ("index bits, log2 of the span", "((uint64_t)1 << b) < (uint64_t)span + 1", "((uint64_t)1 << b) < (uint64_t)span"),
    ("index packing, shifted stream", "uint64_t bit = k * (uint64_t)bits + (uint64_t)b;\n            if ((v >> b) & 1u)",
     "uint64_t bit = k * (uint64_t)bits + (uint64_t)b + 1;\n            if ((v >> b) & 1u)"),
    ("quantization, 65536 levels", "v = rint(65535.0 * (", "v = rint(65536.0 * ("),
    ("dequantization, lo dropped", "pos[3 * i + a] = fmaf((float)q[3 * i + a], step[a], lo[a]);",
     "pos[3 * i + a] = fmaf((float)q[3 * i + a], step[a], 0.0f);"),
    ("ray cast, facing sign", "if (!(det > 0.0f)) continue;", "if (!(det < 0.0f)) continue;"),
    ("ray cast, near test dropped", "t >= nearv)) continue;", "t >= 0.0f)) continue;"),
    ("ray cast, b0 from u twice", "            b0 = b0 - w;\n            float t", "            b0 = b0 - u;\n            float t"),
    ("ray cast, depth from e1", "float t = dot3(e2, qv) / det;", "float t = dot3(e1, qv) / det;"),
    ("ray cast routing, s2 threshold", "> (int64_t)s2_max) {", ">= (int64_t)s2_max) {"),
    ("mip rays, left neighbour", "ray_bary(v, cam, cp, x + (q & 1), y + (q >> 1), b);",
     "ray_bary(v, cam, cp, x - (q & 1), y + (q >> 1), b);"),
    ("mip rays, no top neighbour", "ray_bary(v, cam, cp, x + (q & 1), y + (q >> 1), b);",
     "ray_bary(v, cam, cp, x + (q & 1), y, b);"),
    ("mip level rounded", "lev = isfinite(F) ? floor_log2f(F) : tx->log2_size;",
     "lev = isfinite(F) ? (int)rintf(log2f(F)) : tx->log2_size;"),
    ("mip footprint from u only", "float F = fmaxf(du, dv) * (float)(1 << tx->log2_size);",
     "float F = du * (float)(1 << tx->log2_size);"),
    ("texel row and column swapped", "uint64_t texel = off + (uint64_t)cv * (uint64_t)side + (uint64_t)cu;",
     "uint64_t texel = off + (uint64_t)cu * (uint64_t)side + (uint64_t)cv;"),
    ("mip level offset", "        off += sl * sl;\n", "        off += sl;\n"),
    ("texture v from u", "tx->uv[2 * (uint64_t)vi[1] + 1]", "tx->uv[2 * (uint64_t)vi[1]]"),
    ("texel from the right neighbour's uv", "float cu = floorf(us[0] * fs);", "float cu = floorf(us[1] * fs);"),
    ("clip, near-plane w interpolated", "    if (p == 0) r.w = nearv;\n    else if (r.w < nearv) r.w = nearv;",
     "    if (r.w < nearv) r.w = nearv;"),
    ("ray cast routing, extent rule dropped", "int large = mxx - mnx >= 16384 || mxy - mny >= 16384 ||",
     "int large = 0 ||"),
]

PY_MUTATIONS = [
    ("adjoint, sign of the first term", "dv = ((gam[:, jm] - gbar)[:, None] * np.cross(v[jp], r)",
     "dv = ((gam[:, jm] - gbar)[:, None] * np.cross(r, v[jp])"),
    ("adjoint, gbar dropped", "              + (gam[:, jp] - gbar)[:, None]", "              + (gam[:, jp])[:, None]"),
    ("adjoint, dpos without M^T", "np.add.at(dpos, I[:, j], dv @ M[:, :3])", "np.add.at(dpos, I[:, j], dv)"),
    ("adjoint, dcol to the wrong vertex", "np.add.at(dcol, I[:, k], g * b[:, k:k + 1])",
     "np.add.at(dcol, I[:, (k + 1) % 3], g * b[:, k:k + 1])"),
    ("forward64, ray y scaled by fx", "    r[..., 1] = (ndy / fy)[:, None]", "    r[..., 1] = (ndy / fx)[:, None]"),
]

CASES = [("oracle/curast_oracle.c",) + m for m in C_MUTATIONS] + [("oracle/adjoint.py",) + m for m in PY_MUTATIONS]


def _copy_tree(dst):
    ign = shutil.ignore_patterns("_build", "__pycache__")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ign)
    shutil.copytree(os.path.join(ROOT, "synthetic"), os.path.join(dst, "synthetic"), ignore=ign)
    os.makedirs(os.path.join(dst, "tests"))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))


def _run_case(base, k, rel, name, old, new):
    d = os.path.join(base, f"m{k:02d}")
    _copy_tree(d)
    path = os.path.join(d, rel)
    with open(path) as f:
        src = f.read()
    if src.count(old) != 1:
        return name, f"mutation site found {src.count(old)} times"
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py"], cwd=d, capture_output=True, text=True, timeout=900)
    return name, None if r.returncode != 0 else "survived every pin"


def test_planted_mistakes_fail_a_pin(tmp_path):
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        futs = [ex.submit(_run_case, str(tmp_path), k, *c) for k, c in enumerate(CASES)]
        results = [f.result() for f in futs]
    bad = [f"{name}: {why}" for name, why in results if why is not None]
    assert not bad, "\n".join(bad)
