"""Strength of the oracle's pins: plant one plausible mistake at a time in a copy
of the oracle (a wrong constant, sign, index or operand; a dropped term), build
that copy on the CPU, and check that the pin suites fail on it.

The golden regression of the small clip is left out of these runs: it compares
the oracle with values the oracle itself wrote, so only the pins tied to
something outside the oracle (closed forms, scipy/numpy routines, brute force,
central differences, the second, float-input implementation of the forward)
count here.  CPU only."""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

# (file, original text, planted text, what the slip is); every site occurs in the file
MUTANTS = [
    ("oracle.c", "I[i] = s / 765.0;", "I[i] = s / 755.0;", "intensity scale"),
    ("oracle.c", "if (10 * s > smax) {", "if (10 * s >= smax) {", "hue threshold boundary"),
    ("oracle.c", "- fabs(rn - gn) / 2.0 - bn);", "+ fabs(rn - gn) / 2.0 - bn);", "yellow channel sign"),
    ("oracle.c", "RG[i] = R - G;", "RG[i] = G - R;", "red-green opponent sign"),
    ("oracle.c", "acc += k[j + 2] * k[i + 2] / 256.0 * in[yy * w + xx];",
     "acc += k[j + 2] * k[i + 2] / 255.0 * in[yy * w + xx];", "REDUCE normalisation"),
    ("oracle.c", "  static const double k[5] = {1.0, 4.0, 6.0, 4.0, 1.0};\n  int h2 = (h + 1) / 2",
     "  static const double k[5] = {1.0, 4.0, 6.0, 4.0, 1.0};\n  int h2 = h / 2", "REDUCE output height"),
    ("oracle.c", "kre[(v + radius) * n + (u + radius)] = g * (cos(ph) - kr) / sg;",
     "kre[(v + radius) * n + (u + radius)] = g * cos(ph) / sg;", "Gabor zero-mean term dropped"),
    ("oracle.c", "u * cos(theta) + v * sin(theta)", "v * cos(theta) + u * sin(theta)", "Gabor axes transposed"),
    ("oracle.c", "      out[y * w + x] = sqrt(re * re + im * im);\n    }\n}\n\n/* Across",
     "      out[y * w + x] = fabs(re);\n    }\n}\n\n/* Across", "Gabor energy without the odd part"),
    ("oracle.c", "double sy = mind(maxd((y + 0.5) * hs / (double)hd - 0.5, 0.0), hs - 1.0);",
     "double sy = mind(maxd(y * hs / (double)hd, 0.0), hs - 1.0);", "upsample without half-pixel centres"),
    ("oracle.c", "double mbar = nt > 1 ? (sum - 1.0) / (nt - 1) : 0.0;",
     "double mbar = nt > 1 ? sum / nt : 0.0;", "N(.) mean keeps the global maximum"),
    ("oracle.c", "double f = (1.0 - mbar) * (1.0 - mbar);", "double f = (1.0 - mbar);", "N(.) factor not squared"),
    ("oracle.c", "map[i] = fabs(opp ? cen[i] + up[i] : cen[i] - up[i]);",
     "map[i] = fabs(cen[i] - up[i]);", "opponent center-surround sign"),
    ("oracle.c", "S[i] += P->w[k] * tmp[i];", "S[i] += tmp[i];", "conspicuity weights dropped"),
    ("oracle.c", "orc_gabor_kernel(k * M_PI / no,", "orc_gabor_kernel(k * M_PI / (2 * no),", "orientation spacing"),
    ("oracle.c", "*w_f = a / (a + b + P_prev);", "*w_f = b / (a + b + P_prev);", "Kalman gain numerator"),
    ("oracle.c", "return a * (b + P_prev) / (a + b + P_prev);", "return a * b / (a + b + P_prev);",
     "Kalman variance recursion"),
    ("oracle.c", "double qi = edge ? P->eps : (mx > 0 ? saliency[i] / mx : 0.0);",
     "double qi = mx > 0 ? saliency[i] / mx : 0.0;", "frame-edge prior dropped"),
    ("oracle.c", "prior[i] = (f ? w_f * f[i] : 0.0) + (1.0 - w_f) * qi;",
     "prior[i] = (f ? w_f * f[i] : 0.0) + qi;", "prior not a convex combination"),
    ("oracle.c", "cov[a][k][j] = c[k][j] / sw + (k == j ? 1e-4 : 0.0);", "cov[a][k][j] = c[k][j] / sw;",
     "covariance ridge dropped"),
    ("oracle.c", "double w = a ? prior[i] : 1.0 - prior[i];", "double w = a ? 1.0 - prior[i] : prior[i];",
     "label weights swapped"),
    ("oracle.c", "lconst[a] = 0.5 * log(det3(cov[a]))", "lconst[a] = log(det3(cov[a]))", "log-determinant factor"),
    ("oracle.c", "for (int j = 0; j < 3; ++j) q += d[k] * icov[a][k][j] * d[j];",
     "for (int j = 0; j < 3; ++j) q += d[k] * icov[a][j][j] * d[j];", "Mahalanobis index"),
    ("oracle.c", "cs[i] = quantize(P->cap_scale, D[0] - m);\n    ct[i] = quantize(P->cap_scale, D[1] - m);",
     "cs[i] = quantize(P->cap_scale, D[1] - m);\n    ct[i] = quantize(P->cap_scale, D[0] - m);", "terminals swapped"),
    ("oracle.c", "exp(-dI * dI / (2.0 * P->sigma_I * P->sigma_I)) / dist;",
     "exp(-dI * dI / (2.0 * P->sigma_I * P->sigma_I));", "n-link distance dropped"),
    ("oracle.c", "c = orc_ncap_value(P, s1 - s2, k >= 2);", "c = orc_ncap_value(P, s1 - s2, k >= 1);",
     "diagonal flag on a vertical link"),
    ("oracle.c", "double v = floor(K * x + 0.5);", "double v = floor(K * x);", "capacity rounding"),
    ("oracle.c", "e += mask[v] ? ct[v] : cs[v];", "e += mask[v] ? cs[v] : ct[v];", "cut energy terminals"),
    ("oracle.c", "if (g.r[a] > 0 && !mask[g.head[a]]) {", "if (g.r[a ^ 1] > 0 && !mask[g.head[a]]) {",
     "BK source set along reverse residuals"),
    ("oracle.c", "tr[v] = (int64_t)cs[v] - ct[v];", "tr[v] = (int64_t)ct[v] - cs[v];", "BK terminal residual sign"),
    ("oracle.c", "mask[v] = par[v] != -2;", "mask[v] = par[v] == -2;", "EK source set complemented"),
    ("oracle.c", "g_add(g, y * W + x, yy * W + xx, c, c);", "g_add(g, y * W + x, yy * W + xx, c, 0);",
     "n-links one-way"),
    ("oracle.c", "NB_DX[4] = {1, 0, 1, -1}", "NB_DX[4] = {1, 0, 1, 1}", "second diagonal offset"),
    ("oracle.c", "for (int l = 0; l < level; ++l) n = (n + 1) / 2;", "for (int l = 0; l < level; ++l) n = n / 2 + 1;",
     "level size rounding"),
    ("oracle.c", "out[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) / d;",
     "out[1][2] = (m[0][0] * m[1][2] - m[0][2] * m[1][0]) / d;", "3x3 inverse cofactor sign"),
    ("oracle.c", "m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);\n}",
     "m[0][2] * (m[1][1] * m[2][0] - m[1][0] * m[2][1]);\n}", "3x3 determinant term sign"),
    ("oracle.c", "logp[m] = log(g->pi[m]) - 0.5 * q", "logp[m] = -0.5 * q", "mixture weight dropped"),
    ("oracle.c", "q += dv[k] * Ai[k][j] * dv[j];", "q += dv[k] * Ai[j][j] * dv[j];", "mixture Mahalanobis index"),
    ("oracle.c", "r[(size_t)i * M + m] = exp(lp[m] - mx) / s;", "r[(size_t)i * M + m] = exp(lp[m] - mx);",
     "responsibilities not normalised"),
    ("oracle.c", "g->pi[m] = Nm[m] / Ntot;", "g->pi[m] = 1.0 / M;", "mixture weights never updated"),
    ("oracle.c", "g->cov[m][k][j] = cv[k][j] / Nm[m] + (k == j ? 1e-4 : 0.0);",
     "g->cov[m][k][j] = cv[k][j] / sw + (k == j ? 1e-4 : 0.0);", "component covariance normaliser"),
    ("oracle.c", "for (int k = 0; k < 3; ++k) mu[k] /= Nm[m];", "for (int k = 0; k < 3; ++k) mu[k] /= sw;",
     "component mean normaliser"),
    ("oracle.c", "int nty = (h + tile - 1) / tile, ntx = (w + tile - 1) / tile;",
     "int nty = h / tile, ntx = w / tile;", "N(.) partial edge tiles dropped"),
    ("oracle.c", "for (int u = -radius; u <= radius; ++u) sg += exp(-(u * u + v * v) / (2 * sigma * sigma));",
     "for (int u = -radius; u <= radius; ++u) sg += exp(-(u * u + v * v) / (sigma * sigma));",
     "mask smoothing normaliser"),
    ("oracle.c", "double p = in[clampi(y + v, 0, h - 1) * w + clampi(x + u, 0, w - 1)];",
     "double p = in[clampi(y + u, 0, h - 1) * w + clampi(x + v, 0, w - 1)];", "Gabor applied transposed"),
    ("oracle.c", "double fx = sx - x0;", "double fx = x1 - sx;", "upsample weight side"),
    ("oracle.c", "for (int k = 0; k < 3; ++k) mu[a][k] = m[k] / sw;", "for (int k = 0; k < 3; ++k) mu[a][k] = m[k] / n;",
     "colour mean normaliser"),
    ("oracle.c", "double xi = -log(mind(maxd(p, eps), 1.0 - eps));", "double xi = -log(maxd(p, eps));",
     "prior clamp at 1 - eps dropped"),
    ("oracle.c", "    *w_f = 0.0;\n    return a;", "    *w_f = 0.0;\n    return a + b;", "first-frame variance"),
    ("oracle.c", "    if (tr[x] < delta) delta = tr[x];\n", "\n", "BK bottleneck ignores the source arc"),
    ("oracle.c", "flow += m; /* s -> v -> t directly */", "/* s -> v -> t dropped */", "BK direct terminal flow"),
    ("oracle.c", "  memcpy(st->prev_mask, mask, n);\n  st->P = Pt;", "  st->P = Pt;", "previous mask never carried over"),
    ("oracle.c", "  st->P = Pt;\n  st->t += 1;", "  st->t += 1;", "Kalman variance never carried over"),
    ("oracle.c", "st->t > 0 ? st->prev_mask : NULL, w_f, q, prior);", "NULL, w_f, q, prior);",
     "previous segmentation ignored by the prior"),
    ("oracle.c", "int64_t cut = orc_maxflow_bk(H, W, P->neighbourhood, cs, ct, nc, mask);",
     "int64_t cut = orc_maxflow_bk(H, W, 4, cs, ct, nc, mask);", "frame cut on the wrong neighbourhood"),
    ("oracle.c", "  if (v > 16777216.0) v = 16777216.0;\n", "\n", "capacity cap at 2^24 dropped"),
    ("oracle.c", "if (!(mx - mn > flat)) {", "if (!(mx - mn > 10.0 * flat)) {", "N(.) flat-map threshold"),
    ("oracle.c", "orc_normalize(hS, wS, acc + (size_t)(3 + k) * nS, P->norm_tile, P->norm_flat, tmp);",
     "memcpy(tmp, acc + (size_t)(3 + k) * nS, sizeof(double) * nS);", "per-orientation N(.) dropped"),
    ("oracle.c", "orc_normalize(hl[c], wl[c], map, P->norm_tile, P->norm_flat, nm);",
     "memcpy(nm, map, sizeof(double) * nc);", "feature-map N(.) dropped"),
    ("oracle.c", "const double* sur = f < 3 ? X[f][s] : Ot[f - 3][s];",
     "const double* sur = f < 3 ? X[f][s] : X[0][s];", "orientation surround from the intensity pyramid"),
    ("oracle.c", "orc_normalize(hS, wS, C[k], P->norm_tile, P->norm_flat, tmp);",
     "memcpy(tmp, C[k], sizeof(double) * nS);", "conspicuity N(.) dropped"),
    ("oracle.c", "for (int l = c; l < sS; ++l) {", "for (int l = c + 1; l < sS; ++l) {",
     "one REDUCE too few to sigma_S"),
    ("oracle.c", "      s += w[i] * d2;\n      for (int k = 0; k < 3; ++k) acc[k] += w[i] * d2 * c[k];",
     "      s += w[i] * sqrt(d2);\n      for (int k = 0; k < 3; ++k) acc[k] += w[i] * sqrt(d2) * c[k];",
     "k-means seeds weighted by D instead of D^2"),
    ("oracle.c", "        for (int k = 0; k < 3; ++k) ctr[m][k] = S[m][k] / W[m];\n  }", "        ;\n  }",
     "Lloyd centers never move"),
    ("oracle.c", "    g->pi[m] = W[m] / sw;", "    g->pi[m] = 1.0 / M;", "k-means start with uniform weights"),
    ("oracle.c", "P->gmm_update && st->gmm_valid && st->t > 0);", "0);", "previous frame's mixtures ignored"),
    ("oracle.c", "      if (mix) mix[a] = gm[a];", "", "fitted mixtures not carried to the next frame"),
    ("oracle_grad.c", "+= KB[j + 2] * KB[i + 2] * g_out[y * w2 + x];", "+= KB[j + 2] * g_out[y * w2 + x];",
     "REDUCE adjoint drops a tap factor"),
    ("oracle_grad.c", "double dm = sgv * (-2.0 * (1 - st->mbar)) / (st->nt - 1);",
     "double dm = sgv * (-2.0 * (1 - st->mbar)) / st->nt;", "N(.) adjoint tile-mean count"),
    ("oracle_grad.c", "smin += gp[i] * (vp - 1) / D;", "smin += gp[i] * vp / D;", "N(.) adjoint of the minimum"),
    ("oracle_grad.c", "kre[(v + R) * n + (u + R)] * gr + kim[(v + R) * n + (u + R)] * gi;",
     "kre[(v + R) * n + (u + R)] * gr - kim[(v + R) * n + (u + R)] * gi;", "Gabor adjoint odd-part sign"),
    ("oracle_grad.c", "double t = (grn * r + ggn * g + gbn * b) * 3.0 / (s * s);",
     "double t = (grn * r + ggn * g + gbn * b) * 3.0 / s;", "hue normalisation adjoint power"),
    ("oracle_grad.c", "double gs = gI[i] / 765.0,", "double gs = gI[i] / 255.0,", "intensity adjoint scale"),
    ("oracle_grad.c", "double aY = fmin(r, g) - b > 0;", "double aY = fmax(r, g) - b > 0;", "yellow clamp decision"),
    ("oracle_grad.c", "wr = -Q * dr / (den * den);", "wr = Q * dr / (den * den);", "Kalman gain tangent sign"),
    ("oracle_grad.c", "Pr = (Q * dr * den - num * dr) / (den * den);", "Pr = (Q * dr * den + num * dr) / (den * den);",
     "Kalman variance tangent sign"),
    ("oracle_grad.c", "g_src[y0 * ws + x1] += (1 - fy) * fx * g;", "g_src[y0 * ws + x1] += (1 - fy) * (1 - fx) * g;",
     "upsample adjoint weight"),
]

# A slip in the forward oracle must fail a pin of test_oracle_pins.py (tied to closed forms,
# library routines and brute force), not only the agreement of the forward with the backward
# oracle's second forward implementation; a slip in the backward oracle must fail
# test_oracle_grad.py (central differences and closed forms of the adjoints).
PIN_TESTS = {"oracle.c": [os.path.join(ROOT, "tests", "test_oracle_pins.py")],
             "oracle_grad.c": [os.path.join(ROOT, "tests", "test_oracle_grad.py")]}


def _build_mutant(tmp, fname, old, new):
    for f in ("oracle.c", "oracle_grad.c", "oracle.h"):
        shutil.copy(os.path.join(ORACLE, f), os.path.join(tmp, f))
    path = os.path.join(tmp, fname)
    with open(path) as f:
        src = f.read()
    assert old in src, f"planted-mistake site not found in {fname}: {old!r}"
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(tmp, "liboracle.so")
    subprocess.run(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-w", "-o", lib,
                    os.path.join(tmp, "oracle.c"), os.path.join(tmp, "oracle_grad.c"), "-lm"], check=True)
    return lib


def _pins_on(lib, fname):
    # the concurrent runs share the source tree: none of them writes bytecode there
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=lib, PYTHONDONTWRITEBYTECODE="1")
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", *PIN_TESTS[fname], "-x", "-q", "-p", "no:cacheprovider",
                            "-k", "not regression_golden"], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=300)
    except subprocess.TimeoutExpired:
        return "timeout", ""
    return r.returncode, r.stdout[-400:]


def test_every_planted_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as base:
        def one(i):
            fname, old, new, what = MUTANTS[i]
            tmp = os.path.join(base, str(i))
            os.mkdir(tmp)
            return what, _pins_on(_build_mutant(tmp, fname, old, new), fname)

        with ThreadPoolExecutor(max_workers=min(4, os.cpu_count() or 1)) as ex:
            results = list(ex.map(one, range(len(MUTANTS))))
    # exit code 1: a pin failed.  0 would mean every pin passed; anything else (pytest
    # unable to run, a crashed process) is not counted as a catch either
    survivors = [(what, rc, tail) for what, (rc, tail) in results if rc != 1]
    assert not survivors, survivors


def test_the_unmodified_copy_passes_the_pins():
    with tempfile.TemporaryDirectory() as tmp:
        lib = _build_mutant(tmp, "oracle.c", "I[i] = s / 765.0;", "I[i] = s / 765.0;")
        for fname in PIN_TESTS:
            rc, tail = _pins_on(lib, fname)
            assert rc == 0, tail
