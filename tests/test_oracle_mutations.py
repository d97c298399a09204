"""The pins catch plausible mistakes in the oracle (CPU).

Each of the 85 cases below plants one mistake in a copy of oracle/dts_oracle.c — a dropped term, a wrong
sign, index or operand, passes in the wrong order — compiles the copy with the oracle's own
flags, and runs the pin suite (tests/test_oracle_pins.py) against it in a fresh process
(DTS_ORACLE_SO points the oracle package at the copy).  Every mutant must fail at least one pin;
the unmutated copy, built the same way, must pass them all.  The mistakes are planted in the
oracle only, on the CPU.
"""
import concurrent.futures
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dts_oracle.c")

# (name, text in dts_oracle.c, replacement): each text occurs exactly once
MUTANTS = [
    ("schedule: passes in reverse order", "pow(2.0, (double)(N - i))", "pow(2.0, (double)(i - 1))"),
    ("schedule: sqrt(2) dropped from a_i", "a[i - 1] = exp(-sqrt(2.0) / s);", "a[i - 1] = exp(-1.0 / s);"),
    ("distances: L1 without the 1", "dX[p] = (norm == ORC_NORM_L2) ? sqrt(1.0 + k * k * s) : 1.0 + k * s;",
     "dX[p] = (norm == ORC_NORM_L2) ? sqrt(1.0 + k * k * s) : k * s;"),
    ("distances: dY from the left neighbour", "double diff = I[c * plane + p] - I[c * plane + p - W];",
     "double diff = I[c * plane + p] - I[c * plane + p - 1];"),
    ("distances: L2 with k for k^2", "dY[p] = (norm == ORC_NORM_L2) ? sqrt(1.0 + k * k * s)",
     "dY[p] = (norm == ORC_NORM_L2) ? sqrt(1.0 + k * s)"),
    ("causal sweep: weights swapped", "u[j * su] = (1.0 - w) * u[j * su] + w * u[(j - 1) * su];",
     "u[j * su] = w * u[j * su] + (1.0 - w) * u[(j - 1) * su];"),
    ("anti-causal sweep: d[j] for d[j+1]", "double w = pow(a, d[(j + 1) * sd]);\n        u[j * su]",
     "double w = pow(a, d[j * sd]);\n        u[j * su]"),
    ("filter: vertical pass first", "orc_row_pass(H, W, dst, dX, a[i]);\n        orc_col_pass(H, W, dst, dY, a[i]);",
     "orc_col_pass(H, W, dst, dY, a[i]);\n        orc_row_pass(H, W, dst, dX, a[i]);"),
    ("filter: vertical pass with another pass's a", "orc_col_pass(H, W, dst, dY, a[i]);",
     "orc_col_pass(H, W, dst, dY, a[N - 1 - i]);"),
    ("gradient step: smoothness term sign", "out[p] = zk[p] - e * (lambda * (zk[p] - zbar[p])",
     "out[p] = zk[p] - e * (lambda * (zbar[p] - zk[p])"),
    ("fixed point: z_k for z_bar", "(lambda * zbar[p] + cw * t[p]) / den", "(lambda * zk[p] + cw * t[p]) / den"),
    ("Charbonnier: eps not squared", "r / sqrt(r * r + eps * eps) : r;", "r / sqrt(r * r + eps) : r;"),
    ("support: own weight counted twice", "out[j * so] = P[j] + Q[j] - x[j * sx];", "out[j * so] = P[j] + Q[j];"),
    ("Eq. 7: variance without the square", "double v = m2[i] - m1[i] * m1[i];", "double v = m2[i] - m1[i];"),
    ("box kernel: radius without sqrt(3)", "const double r = sigma[i] * sqrt(3.0);", "const double r = sigma[i];"),
    ("adjoint: sign of ln a", "double la = log(a);", "double la = -log(a);"),
    ("adjoint: causal weight gradient sign", "wbar[j] += gJ[j] * (J[j - 1] - x[j * sx]);",
     "wbar[j] += gJ[j] * (x[j * sx] - J[j - 1]);"),
    ("backward, fixed point: confidence gradient sign",
     "const double gcw = lambda * (t[p] - zbar[p]) / (den * den) * g[p];",
     "const double gcw = lambda * (zbar[p] - t[p]) / (den * den) * g[p];"),
    ("fixed point, Charbonnier: loss weight left out", "cw = chat[p] / sqrt(r * r + eps * eps);", "cw = chat[p];"),
    ("fixed point, Charbonnier: weight squared", "cw = chat[p] / sqrt(r * r + eps * eps);",
     "cw = chat[p] / (r * r + eps * eps);"),
    ("backward, fixed point Charbonnier: iterate path dropped", "gprev[p] = gr;", "gprev[p] = 0.0;"),
    ("backward, fixed point Charbonnier: target path sign", "tb[p] += cw / den * g[p] - gr;",
     "tb[p] += cw / den * g[p] + gr;"),
    ("backward, fixed point Charbonnier: weight derivative power", "-c[p] * r * w * w * w * gcw",
     "-c[p] * r * w * w * gcw"),
    ("backward, fixed point Charbonnier: confidence gradient without the weight", "cb[p] += w * gcw;",
     "cb[p] += gcw;"),
    ("backward, gradient step: data term dropped from the carry",
     "gprev[p] = (1.0 - eta * lambda - eta * c[p] * d2) * g[p];", "gprev[p] = (1.0 - eta * lambda) * g[p];"),
    ("CG: factor 2 of the data term dropped", "q[i] = lambda * (t1[i] - t2[i]) + 2.0 * c[i] * p[i];",
     "q[i] = lambda * (t1[i] - t2[i]) + c[i] * p[i];"),
    ("CG: beta inverted", "const double beta = rr_new / rr;", "const double beta = rr / rr_new;"),
    ("guide gradient: left neighbour sign", "Gc[p - 1] -= g;", "Gc[p - 1] += g;"),
    ("guide gradient, L2: k for k^2", "? dXbar[p] * k * k * diff / dX[p]", "? dXbar[p] * k * diff / dX[p]"),
    ("schedule: sqrt(3) dropped from sigma_i", "double s = sigma_s * sqrt(3.0) * pow(", "double s = sigma_s * pow("),
    ("support weighting: ratio inverted", "chat[p] = c[p] * sf / chat[p];", "chat[p] = c[p] * chat[p] / sf;"),
    ("support: flat-guide value not squared", "*s_flat = ((1.0 + a) / (1.0 - a)) * ((1.0 + a) / (1.0 - a));",
     "*s_flat = ((1.0 + a) / (1.0 - a));"),
    ("support: anti-causal d[j] for d[j+1]", "pow(a, d[(j + 1) * sd]) * Q[j + 1]", "pow(a, d[j * sd]) * Q[j + 1]"),
    ("Eq. 7: 2 sigma_c^2 without the 2", "c[i] = exp(-v / (2.0 * sigma_c * sigma_c));", "c[i] = exp(-v / (sigma_c * sigma_c));"),
    ("box kernel: coordinate from the previous distance", "ct[j] = ct[j - 1] + d[j * sd];",
     "ct[j] = ct[j - 1] + d[(j - 1) * sd];"),
    ("adjoint: anti-causal weight gradient sign", "wbar[j + 1] += h[j] * (Kv[j + 1] - J[j]);",
     "wbar[j + 1] += h[j] * (J[j] - Kv[j + 1]);"),
    ("adjoint: anti-causal input factor", "h[j] = (1.0 - w[j + 1]) * h[j];", "h[j] = w[j + 1] * h[j];"),
    ("filter adjoint: row passes with another pass's a",
     "row_pass_adjoint(H, W, U + (long)p * n, dX, a[p / 2], g, g2, dXbar);",
     "row_pass_adjoint(H, W, U + (long)p * n, dX, a[N - 1 - p / 2], g, g2, dXbar);"),
    ("backward, gradient step: confidence dropped from the target gradient", "tb[p] += eta * c[p] * d2 * g[p];",
     "tb[p] += eta * d2 * g[p];"),
    ("backward: the z_0 = t path dropped", "for (long p = 0; p < n; ++p) tb[p] += g[p];", ";"),
    ("CG: initial residual without the factor 2", "r[i] = 2.0 * c[i] * t[i] - q[i];", "r[i] = c[i] * t[i] - q[i];"),
    ("causal sweep: first step skipped", "for (int j = 1; j < n; ++j) {\n        double w = pow(a, d[j * sd]);",
     "for (int j = 2; j < n; ++j) {\n        double w = pow(a, d[j * sd]);"),
    ("anti-causal sweep: last step skipped",
     "for (int j = n - 2; j >= 0; --j) {\n        double w = pow(a, d[(j + 1) * sd]);",
     "for (int j = n - 3; j >= 0; --j) {\n        double w = pow(a, d[(j + 1) * sd]);"),
    ("support weighting: step limit inverted", "1.0 / (lambda + chat[p]) < e) e =", "1.0 / (lambda + chat[p]) > e) e ="),
    ("box kernel: average over one sample too many", "tmp[i] = sum / cnt;", "tmp[i] = sum / (cnt + 1);"),
    ("distances: dY without the absolute value",
     "double diff = I[c * plane + p] - I[c * plane + p - W];\n                    s += (norm == ORC_NORM_L2) ? diff * diff : fabs(diff);",
     "double diff = I[c * plane + p] - I[c * plane + p - W];\n                    s += (norm == ORC_NORM_L2) ? diff * diff : diff;"),
    ("box kernel: columns on dX", "box_line(H, dst + x, W, dY + x, W, r, ct, tmp);",
     "box_line(H, dst + x, W, dX + x, W, r, ct, tmp);"),
    ("adjoint: first input gradient dropped", "gin[0] = gJ[0];", "gin[0] = 0.0;"),
    ("backward, fixed point: lambda for c in the target gradient", "tb[p] += cw / den * g[p] - gr;",
     "tb[p] += lambda / den * g[p] - gr;"),
    ("backward, Charbonnier: curvature", "eps * eps / (s * s * s)", "eps / (s * s)"),
    ("CG: alpha inverted", "const double alpha = rr / pq;", "const double alpha = pq / rr;"),
    ("CG: residual updated with p", "r[i] -= alpha * q[i];", "r[i] -= alpha * p[i];"),
    ("support: distance ignored", "P[j] = x[j * sx] + pow(a, d[j * sd]) * P[j - 1];", "P[j] = x[j * sx] + a * P[j - 1];"),
    ("guide gradient, dY: wrong neighbour", "Gc[p - W] -= g;", "Gc[p - 1] -= g;"),
    ("schedule: the -1 of 4^N - 1 dropped", "sqrt(pow(4.0, (double)N) - 1.0)", "sqrt(pow(4.0, (double)N))"),
    ("adjoint: carried gradient weighted by w_j", "gJ[j] = h[j] + w[j + 1] * gJ[j + 1];", "gJ[j] = h[j] + w[j] * gJ[j + 1];"),
    ("adjoint: anti-causal gradient carried with w_{j-1}", "h[j] = gout[j * sg] + w[j] * h[j - 1];",
     "h[j] = gout[j * sg] + w[j - 1] * h[j - 1];"),
    ("fixed point: lambda + c = 0 gives 0", "/ den : zk[p];", "/ den : 0.0;"),
    ("backward, fixed point: lambda + c = 0 stops the gradient", "gprev[p] = g[p];", "gprev[p] = 0.0;"),
    ("gradient step: step size ignored", "double e = eta;", "double e = 1.0;"),
    ("distances: sigma_r / sigma_s",
     "double k = sigma_s / sigma_r;\n    long plane = (long)H * W;\n#pragma omp parallel for",
     "double k = sigma_r / sigma_s;\n    long plane = (long)H * W;\n#pragma omp parallel for"),
    ("distances: L2 without the square root", "dX[p] = (norm == ORC_NORM_L2) ? sqrt(1.0 + k * k * s)",
     "dX[p] = (norm == ORC_NORM_L2) ? (1.0 + k * k * s)"),
    ("checkpoints in reverse order", "if (ckpt) memcpy(ckpt + (long)k * n, z,", "if (ckpt) memcpy(ckpt + (long)(K - 1 - k) * n, z,"),
    ("CG: one step fewer", "for (int k = 0; k < K && rr > 0.0; ++k)", "for (int k = 1; k < K && rr > 0.0; ++k)"),
    ("CG: z_init ignored", "memcpy(z, z0 ? z0 : t, sizeof(double) * (size_t)n);\n    cg_apply_M",
     "memcpy(z, t, sizeof(double) * (size_t)n);\n    cg_apply_M"),
    ("filter adjoint: pass inputs recomputed in the wrong direction",
     "if (p % 2 == 0)\n            orc_row_pass(H, W, U + (long)(p + 1) * n, dX, a[p / 2]);",
     "if (p % 2 == 1)\n            orc_row_pass(H, W, U + (long)(p + 1) * n, dX, a[p / 2]);"),
    ("gradient step: z_bar halved", "lambda * (zk[p] - zbar[p]) + chat[p]", "lambda * (zk[p] - zbar[p] * 0.5) + chat[p]"),
    ("backward, gradient step: lambda dropped from the smoothness gradient", "gbar[p] = eta * lambda * g[p];",
     "gbar[p] = eta * g[p];"),
    ("backward: z_bar not recomputed", "orc_filter(H, W, dX, dY, N, a, zk, zbar);\n        for (long p = 0; p < n; ++p) {",
     "memcpy(zbar, zk, sizeof(double) * (size_t)n);\n        for (long p = 0; p < n; ++p) {"),
    ("guide gradient, L1: k dropped", ": dXbar[p] * k * ((diff > 0) - (diff < 0));", ": dXbar[p] * ((diff > 0) - (diff < 0));"),
    ("Eq. 7: variance squared", "c[i] = exp(-v / (2.0 * sigma_c * sigma_c));", "c[i] = exp(-v * v / (2.0 * sigma_c * sigma_c));"),
    ("Eq. 7: the mean of t for the mean of t^2", "orc_filter(H, W, dX, dY, N, a, t2, m2);",
     "orc_filter(H, W, dX, dY, N, a, t, m2);"),
    ("Eq. 7: small variances dropped", "if (v < 0.0) v = 0.0;", "if (v < 1e-3) v = 0.0;"),
    ("support: columns on dX", "support_line(H, s + x, W, S + x, W, dY + x, W, a, P, Q);",
     "support_line(H, s + x, W, S + x, W, dX + x, W, a, P, Q);"),
    ("support: anti-causal sum starts at 0", "Q[n - 1] = x[(n - 1) * sx];", "Q[n - 1] = 0.0;"),
    ("support: causal sum starts at 0", "P[0] = x[0];", "P[0] = 0.0;"),
    ("box kernel: window without the absolute value", "if (fabs(ct[m] - ct[i]) <= r) {", "if ((ct[m] - ct[i]) <= r) {"),
    ("Charbonnier: taken for eps = 0 too", "return eps > 0.0 ? r / sqrt(r * r + eps * eps) : r;",
     "return eps >= 0.0 ? r / sqrt(r * r + eps * eps) : r;"),
    ("guide gradient, L2, dY: distance not divided out", "? dYbar[p] * k * k * diff / dY[p]", "? dYbar[p] * k * k * diff"),
    ("backward, Charbonnier: r for rho'(r) in the confidence gradient", "cb[p] -= eta * d1 * g[p];",
     "cb[p] -= eta * r * g[p];"),
    ("filter adjoint: first pass skipped", "for (int p = 2 * N - 1; p >= 0; --p) {", "for (int p = 2 * N - 1; p >= 1; --p) {"),
    ("guide gradient, dY: own pixel sign", "Gc[p] += g;\n                    Gc[p - W] -= g;",
     "Gc[p] -= g;\n                    Gc[p - W] -= g;"),
    ("CG: (I - A) p with the wrong sign", "t1[i] = p[i] - t1[i];", "t1[i] = t1[i] - p[i];"),
    ("backward, gradient step: target gradient sign", "tb[p] += eta * c[p] * d2 * g[p];", "tb[p] -= eta * c[p] * d2 * g[p];"),
    ("backward, gradient step: smoothness sign in the carry",
     "gprev[p] = (1.0 - eta * lambda - eta * c[p] * d2) * g[p];",
     "gprev[p] = (1.0 + eta * lambda - eta * c[p] * d2) * g[p];"),
]


def _build_and_run_pins(tmp, tag, source):
    c_path = os.path.join(tmp, f"{tag}.c")
    so_path = os.path.join(tmp, f"{tag}.so")
    with open(c_path, "w") as f:
        f.write(source)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", so_path,
                    c_path, "-lm"], check=True)
    env = dict(os.environ, DTS_ORACLE_SO=so_path, OMP_NUM_THREADS="1")
    # the copy must load and run before its pin results mean anything (a library that fails to
    # load would fail the pins too)
    probe = subprocess.run([sys.executable, "-c", "import oracle, numpy as np; "
                            "assert oracle.distances(np.zeros((1, 2, 2)), 1.0, 1.0)[0].shape == (2, 2)"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    if probe.returncode != 0:
        return -1000 - probe.returncode, probe.stderr[-2000:]
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    original = open(SRC).read()
    jobs = [("control", original)]
    for k, (name, old, new) in enumerate(MUTANTS):
        assert original.count(old) == 1, f"{name}: the planted text must occur exactly once"
        jobs.append((f"m{k:02d}", original.replace(old, new)))
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda j: _build_and_run_pins(str(tmp_path), *j), jobs))
    rc, out = results[0]
    assert rc == 0, f"the unmutated oracle must pass the pins:\n{out}"
    # pytest exits with 1 when tests ran and some failed; anything else (a load or collection
    # error, a crash) would not show that a pin caught the mistake
    broken = [(MUTANTS[k][0], rc, out) for k, (rc, out) in enumerate(results[1:]) if rc not in (0, 1)]
    assert not broken, f"mutants that did not run the pins: {broken}"
    survivors = [MUTANTS[k][0] for k, (rc, _) in enumerate(results[1:]) if rc == 0]
    assert not survivors, f"mistakes no pin catches: {survivors}"
