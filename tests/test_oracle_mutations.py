"""The oracle's pins are strong enough to catch plausible mistakes.

Each case plants one mistake in a copy of oracle/sfo.c (a wrong sign, index,
pairing, weight, dropped term, misplaced block, ...), builds the copy on the
CPU, and runs the pin tests of tests/test_oracle_pins.py,
tests/test_oracle_maps.py and tests/test_oracle_replay.py against it through
the SFO_LIB override: every mutant must fail at least one pin. The planted
mistakes live only in temporary copies; the oracle itself is not touched.
Mistakes planted in oracle/net.py run against tests/test_oracle_net.py from a
copied tree of their own.
"""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sfo.c")
PIN_FILES = [os.path.join(ROOT, "tests", f) for f in ("test_oracle_pins.py", "test_oracle_maps.py", "test_oracle_replay.py")]

# name -> (text in sfo.c, planted replacement); each text occurs exactly once
MUTANTS = {
    "sign of s in image 1 (Eqs. 1-6)": ("    {+1.0, -1.0, -1.0},\n", "    {-1.0, -1.0, -1.0},\n"),
    "check pair of d_0 swapped": ("{{1, 0}, {3, 2},", "{{0, 1}, {3, 2},"),
    "gradient term dropped from E": ("Eg += psi_grad(", "Eg += 0.0 * psi_grad("),
    "smoothness coupling in the mirrored slot": ("add_block(A, n, slot_of(i2 - i, j2 - j), u, u, -c);",
                                                 "add_block(A, n, slot_of(i - i2, j - j2), u, u, -c);"),
    "bilinear weights of corners 1 and 2 swapped": ("    wts[1] = a * (1 - b);\n    wts[2] = (1 - a) * b;\n",
                                                    "    wts[1] = (1 - a) * b;\n    wts[2] = a * (1 - b);\n"),
    "larger eigenvalue for w_i": ("0.5 * (a + c) - sqrt(", "0.5 * (a + c) + sqrt("),
    "sign of the smoothness rhs": ("b[n * 6 + u] -= c * d;", "b[n * 6 + u] += c * d;"),
    "prolongation without the factor 2": ("2.0 * grid_sample(nxc", "1.0 * grid_sample(nxc"),
    "temporal transfer forward instead of back": ("(double)(i * s) - 2.0 * T_prev[2 * G + n]",
                                                  "(double)(i * s) + 2.0 * T_prev[2 * G + n]"),
    "backtracking accepts any step": ("if (Et <= Ecur) {", "if (Et == Et) {"),
    "W threshold doubled": ("return mx < eps_p ? 1 : 0;", "return mx < 2.0 * eps_p ? 1 : 0;"),
    "F of a level scaled on x only": ("ldexp(1.0, level), ldexp(1.0, level), 1.0", "ldexp(1.0, level), 1.0, 1.0"),
    "halfway image with the sign of s flipped": (
        "double px = x + SIGN[c][0] * f[0] + SIGN[c][1] * f[2] + SIGN[c][2] * f[4];\n"
        "        double py = y + SIGN[c][0] * f[1] + SIGN[c][1] * f[3] + SIGN[c][2] * f[5];\n        acc +=",
        "double px = x - SIGN[c][0] * f[0] + SIGN[c][1] * f[2] + SIGN[c][2] * f[4];\n"
        "        double py = y - SIGN[c][0] * f[1] + SIGN[c][1] * f[3] + SIGN[c][2] * f[5];\n        acc +="),
    "square-root photo block over 2 rho": ("gp[r] * gp[c] / (4.0 * rho_p)", "gp[r] * gp[c] / (2.0 * rho_p)"),
    "square-root gradient block over 2 rho": ("gg[r] * gg[c] / (4.0 * rho_g)", "gg[r] * gg[c] / (2.0 * rho_g)"),
    "IRLS weight without the 1/2": ("p->w_photo / (2.0 * phi(", "p->w_photo / (1.0 * phi("),
    "epipolar Jacobian sign": ("SIGN[il][fld] * Fr[a] + SIGN[ir][fld] * Ftl[a]",
                               "SIGN[il][fld] * Fr[a] - SIGN[ir][fld] * Ftl[a]"),
    "magnitude prior on totals": ("double d = delta[(2 * fld + a) * G + n];", "double d = T[(2 * fld + a) * G + n];"),
    "pyramid filter weight": ("dst[y * w2 + x] = 0.25 * acc;", "dst[y * w2 + x] = 0.3 * acc;"),
    "gradient image without the 1/2": ("gx[y * w + x] = 0.5 * (img[y * w + xp] - img[y * w + xm]);",
                                       "gx[y * w + x] = 1.0 * (img[y * w + xp] - img[y * w + xm]);"),
    "bilinear x derivative with the rows' weights swapped": (
        "*dpx = clx ? 0.0 : (1 - fy) * (p10 - p00) + fy * (p11 - p01);",
        "*dpx = clx ? 0.0 : fy * (p10 - p00) + (1 - fy) * (p11 - p01);"),
    "Jacobi preconditioner dropped": ("Minv[n * 6 + u] = d > 0.0 ? 1.0 / d : 1.0;", "Minv[n * 6 + u] = 1.0;"),
    "Jacobi preconditioner as diag(A) instead of its inverse": ("Minv[n * 6 + u] = d > 0.0 ? 1.0 / d : 1.0;",
                                                                 "Minv[n * 6 + u] = d > 0.0 ? d : 1.0;"),
    "PCG beta inverted": ("double beta = rz_new / rz;", "double beta = rz / rz_new;"),
    "PCG direction from the unpreconditioned residual": (
        "for (int a = 0; a < N; ++a) pv[a] = z[a] + beta * pv[a];",
        "for (int a = 0; a < N; ++a) pv[a] = r[a] + beta * pv[a];"),
    "PCG step length over p.p": ("double alpha = rz / pq;", "double alpha = rz / dot(N, pv, pv);"),
    "backtracking by quarters": ("++bt, t *= 0.5) {", "++bt, t *= 0.25) {"),
    "temporal transfer along the stereo field": ("double X = (double)(i * s) - 2.0 * T_prev[2 * G + n];",
                                                 "double X = (double)(i * s) - 2.0 * T_prev[0 * G + n];"),
    "level F without the Frobenius rescale": ("for (int a = 0; a < 9; ++a) Fl[a] *= sqrt(n0 / n1);",
                                              "for (int a = 0; a < 9; ++a) Fl[a] *= 1.0;"),
    "smoothness system weight from one node": (
        "double c = p->w_reg * p->w_smooth * (wf[n] + wf[m]) * wfl[fld];",
        "double c = p->w_reg * p->w_smooth * 2.0 * wf[n] * wfl[fld];"),
    "magnitude system weight from the smoothness weights": ("double cm = p->w_reg * p->w_mag * mfl[fld];",
                                                            "double cm = p->w_reg * p->w_mag * wfl[fld];"),
    "epipolar pair of time 1 with the wrong left image": ("int il = tt == 0 ? 0 : 2, ir = tt == 0 ? 1 : 3;",
                                                          "int il = tt == 0 ? 0 : 1, ir = tt == 0 ? 1 : 3;"),
    "halfway image as half the sum": ("    return 0.25 * acc;\n}\n\n/* ----", "    return 0.5 * acc;\n}\n\n/* ----"),
    "structure tensor one pixel off the node": ("int qx = i * s + dx, qy = j * s + dy;",
                                                "int qx = i * s + dx + 1, qy = j * s + dy;"),
    "gradient IRLS weight without the 1/2": ("double og = 0.5 * p->w_grad * psi_grad_coef(",
                                             "double og = 1.0 * p->w_grad * psi_grad_coef("),
    "prolongation reads row i/2 for j": ("2.0 * grid_sample(nxc, nyc, Tc + c * Gc, 0.5 * i, 0.5 * j);",
                                         "2.0 * grid_sample(nxc, nyc, Tc + c * Gc, 0.5 * i, 0.5 * i);"),
    "temporal transfer sampled at half the y scale": (
        "grid_sample(nx, ny, delta_prev + c * G, X / s, Y / s);",
        "grid_sample(nx, ny, delta_prev + c * G, X / s, Y / (2 * s));"),
    "gradient term weighted by w_photo in E": ("return p->w_photo * Ep + p->w_grad * Eg + p->w_reg",
                                               "return p->w_photo * Ep + p->w_photo * Eg + p->w_reg"),
    "given W ignored": ("int Wi = Win ? Win[y * w + x] : outlier_weight(e, p->eps_p);",
                        "int Wi = outlier_weight(e, p->eps_p);"),
    "W disagreement margin not measured from eps_p": (
        "if (fabs(mx - p->eps_p) > *margin) *margin = fabs(mx - p->eps_p);", "if (mx > *margin) *margin = mx;"),
    "given cell decision ignored": ("    if (gx >= 0) {", "    if (gx >= 0 && 0) {"),
    "F transposed in the epipolar product": (
        "Fr[a] = Fl[a * 3 + 0] * rr[0] + Fl[a * 3 + 1] * rr[1] + Fl[a * 3 + 2] * rr[2];",
        "Fr[a] = Fl[0 * 3 + a] * rr[0] + Fl[1 * 3 + a] * rr[1] + Fl[2 * 3 + a] * rr[2];"),
    "Schwarz residual sign": ("for (int a = 0; a < N; ++a) r[a] = b[a] - r[a];",
                              "for (int a = 0; a < N; ++a) r[a] = b[a] + r[a];"),
    "Schwarz update not restricted to the tile": (
        "for (int j = tj * tile; j < (tj + 1) * tile && j < ny; ++j)\n"
        "                    for (int i = ti * tile; i < (ti + 1) * tile && i < nx; ++i) {",
        "for (int j = j0; j < j1; ++j)\n                    for (int i = i0; i < i1; ++i) {"),
    "Schwarz subdomain without its overlap": ("int i0 = ti * tile - overlap, j0 = tj * tile - overlap;",
                                               "int i0 = ti * tile, j0 = tj * tile;"),
    "closeness with the wrong sign": ("    return ol - orr;\n", "    return orr - ol;\n"),
    "occlusion tolerance added": ("if (!(closeness(c / 2, f) >= z - tau)) vis = 0;",
                                  "if (!(closeness(c / 2, f) >= z + tau)) vis = 0;"),
    "z-buffer lookup truncates instead of rounding": ("double qx = floor(px + 0.5), qy = floor(py + 0.5);",
                                                      "double qx = floor(px), qy = floor(py);"),
    "second triangle of a cell misplaced": ("int vj[3] = {j, tri == 0 ? j : j + 1, j + 1};",
                                            "int vj[3] = {j, j, j + 1};"),
    "visibility prolongation threshold": ("sfo_sample(wc, hc, P, 0.5 * x, 0.5 * y, NULL, NULL) >= 0.5;",
                                          "sfo_sample(wc, hc, P, 0.5 * x, 0.5 * y, NULL, NULL) > 0.5;"),
    "Gaussian not normalised": ("for (int k = 0; k <= 2 * R; ++k) g[k] /= sum;",
                                "for (int k = 0; k <= 2 * R; ++k) g[k] /= 2.0;"),
    "Gaussian radius 2 sigma": ("int R = (int)ceil(3.0 * sigma);", "int R = (int)ceil(2.0 * sigma);"),
    "illumination correction on the left image": ("val[1][0] -= corr[0];", "val[0][0] -= corr[0];"),
    "box prolongation shifted": ("int xc = x / 2, yc = y / 2;", "int xc = (x + 1) / 2, yc = y / 2;"),
    "stereo residual of time 1 from the wrong check": ("r[N + (size_t)y * w + x] = e[1];",
                                                       "r[N + (size_t)y * w + x] = e[3];"),
}


# planted mistakes in oracle/net.py (the warm-start network), run against tests/test_oracle_net.py
NET_MUTANTS = {
    "input not centred": ("a = np.asarray(imgs, dtype=np.float64) - 0.5", "a = np.asarray(imgs, dtype=np.float64) - 0.0"),
    "output size rounded down": ("return (n + stride - 1) // stride", "return n // stride"),
    "loss gradient without the factor 2": ("g = 2.0 * r / r.size", "g = r / r.size"),
    "input gradient through the flipped kernel": (
        'dxp[sl] += np.einsum("bohw,oc->bchw", dy, w[:, :, u, v])',
        'dxp[sl] += np.einsum("bohw,oc->bchw", dy, w[:, :, 2 - u, 2 - v])'),
    "ReLU gate on the layer's input instead of its output": ("g = g * (pre[k] > 0.0)", "g = g * (acts[k].sum() > 0.0)"),
    "Adam without bias correction": ("mh = mm / (1.0 - beta1 ** t)", "mh = mm"),
    "Adam eps inside the square root": ("x - lr * mh / (np.sqrt(vh) + eps)", "x - lr * mh / np.sqrt(vh + eps)"),
}
NET_SRC = os.path.join(ROOT, "oracle", "net.py")


def _run_net_mutant(name, tmpdir):
    """A copy of the oracle package with the mistake planted in net.py, and the
    network pins run against it from a tree of their own."""
    text, planted = NET_MUTANTS[name]
    src = open(NET_SRC).read()
    assert src.count(text) == 1, f"{name}: anchor text not unique in net.py"
    tag = "".join(ch if ch.isalnum() else "_" for ch in name)
    top = os.path.join(tmpdir, "net_" + tag)
    os.makedirs(os.path.join(top, "oracle"))
    os.makedirs(os.path.join(top, "tests"))
    with open(os.path.join(top, "oracle", "net.py"), "w") as f:
        f.write(src.replace(text, planted))
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), os.path.join(top, "oracle", "__init__.py"))
    for fn in ("conftest.py", "test_oracle_net.py"):
        shutil.copy(os.path.join(ROOT, "tests", fn), os.path.join(top, "tests", fn))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(top, "tests", "test_oracle_net.py"), "-x", "-q",
                        "-p", "no:cacheprovider"], capture_output=True, text=True, env=env, cwd=top)
    return r.returncode, r.stdout[-400:]


def _run_mutant(name, tmpdir):
    text, planted = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(text) == 1, f"{name}: anchor text not unique in sfo.c"
    tag = "".join(ch if ch.isalnum() else "_" for ch in name)
    csrc = os.path.join(tmpdir, f"{tag}.c")
    so = os.path.join(tmpdir, f"{tag}.so")
    with open(csrc, "w") as f:
        f.write(src.replace(text, planted))
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, csrc, "-lm"])
    # one BLAS thread per mutant run: the runs go in parallel
    env = dict(os.environ, SFO_LIB=so, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", *PIN_FILES, "-x", "-q", "-p", "no:cacheprovider"],
                       capture_output=True, text=True, env=env, cwd=ROOT)
    return r.returncode, r.stdout[-400:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    names = sorted(MUTANTS)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = dict(zip(names, ex.map(lambda n: _run_mutant(n, str(tmp_path)), names)))
    missed = [n for n, (rc, _) in results.items() if rc == 0]
    assert not missed, f"mutants that pass every pin: {missed}"
    # a mutant must fail a test, not break the test run itself
    broken = [n for n, (rc, out) in results.items() if rc not in (1,)]
    assert not broken, {n: results[n][1] for n in broken}


def test_every_planted_network_mistake_fails_a_pin(tmp_path):
    names = sorted(NET_MUTANTS)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = dict(zip(names, ex.map(lambda n: _run_net_mutant(n, str(tmp_path)), names)))
    missed = [n for n, (rc, _) in results.items() if rc == 0]
    assert not missed, f"network mutants that pass every pin: {missed}"
    broken = [n for n, (rc, out) in results.items() if rc not in (1,)]
    assert not broken, {n: results[n][1] for n in broken}


def test_the_unmutated_network_copy_passes(tmp_path):
    """The network harness itself: an unchanged copy passes every network pin."""
    NET_MUTANTS["(unchanged)"] = ("import numpy as np", "import numpy as np")
    try:
        rc, out = _run_net_mutant("(unchanged)", str(tmp_path))
    finally:
        del NET_MUTANTS["(unchanged)"]
    assert rc == 0, out


def test_the_unmutated_copy_passes(tmp_path):
    """The harness itself: the oracle built from an unchanged copy passes every pin."""
    so = os.path.join(str(tmp_path), "same.so")
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, SRC, "-lm"])
    r = subprocess.run([sys.executable, "-m", "pytest", *PIN_FILES, "-q", "-p", "no:cacheprovider"],
                       capture_output=True, text=True, env=dict(os.environ, SFO_LIB=so), cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:]
