"""Mutation check of the oracle pins (run by hand; about 20 minutes):

    python tests/mutation_check.py

Plants one plausible mistake at a time -- a flipped sign, a shifted index,
a dropped factor, an exchanged a and b -- in a scratch copy of oracle/, runs
the CPU pins (tests/test_oracle_pins.py, tests/test_khat_scheme.py) against
it, and reports whether some pin fails ("caught"); then the same for the
block GMRES host numerics (csrc/bgmres_host.h against
tests/test_block_host.py).  One mutation is known to survive: a frequency
box two lines narrower changes the discrete rule D only within its
discretisation error; the GPU-versus-oracle parity tests and the regression
fixtures of tests/golden/ fix that choice.  (A shorter kernel truncation
radius used to survive as well; the 4:1 aperture's pin catches it.)
Exit status 1 if any other mutation survives.
"""

import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (file under oracle/, original text, mutated text)
MUTATIONS = [
    ('excitation.py', 'a1 = -kappa0 * st * cf', 'a1 = kappa0 * st * cf'),
    ('excitation.py', 'g1 = (h / q)[:, None] * 2j * (a1', 'g1 = (h / q)[:, None] * -1j * (a1'),
    ('excitation.py', 'g2 = (h / cn)[None, :] * 2j * (a2', 'g2 = (h / cn)[None, :] * -1j * (a2'),
    ('excitation.py', 'g1 = (h / q)[:, None] * 2j * (a1', 'g1 = (h / q)[:, None] * -2j * (a1'),
    ('excitation.py', 'g2 = (h / cn)[None, :] * 2j * (a2', 'g2 = (h / cn)[None, :] * 1j * (a2'),
    ('excitation.py', 'beta = kappa0 * ct', 'beta = -kappa0 * ct'),
    ('excitation.py', 'th_hat = np.array([ct * cf, ct * sf, -st])', 'th_hat = np.array([ct * cf, ct * sf, st])'),
    ('excitation.py', '(a1 * p[2] + beta * p[0])', '(a1 * p[2] - beta * p[0])'),
    ('excitation.py', '(a2 * p[2] + beta * p[1])', '(a2 * p[2] + beta * p[0])'),
    ('excitation.py', 'q[0] = ab / 2.0', 'q[0] = ab / 4.0'),
    ('excitation.py', 'cn[0] = ab / 2.0', 'cn[0] = ab / 4.0'),
    ('excitation.py', 'ex = np.exp(1j * a1 * x)', 'ex = np.exp(-1j * a1 * x)'),
    ('excitation.py', 'return np.outer(cx, sy), np.outer(sx, cy)', 'return np.outer(cx, sy), np.outer(sx, cy).conj()'),
    ('tbc.py', 'val = (1.0 - np.exp(-2j * np.pi * safe * a)) / (2j * np.pi * safe)', 'val = (1.0 - np.exp(2j * np.pi * safe * a)) / (2j * np.pi * safe)'),
    ('tbc.py', "return 0.5 * (em + ep)", "return 0.5 * (em - ep)"),
    ('tbc.py', "return (em - ep) / 2j", "return (em + ep) / 2j"),
    ('tbc.py', "w[0] *= 0.5", "w[0] *= 1.0"),
    ('tbc.py', "return np.exp(2j * np.pi * np.outer(nodes, js) / P)", "return np.exp(-2j * np.pi * np.outer(nodes, js) / P)"),
    ('tbc.py', "self._ex = idft_matrix(np.arange(nx + 1), self.jx, self.Px) / self.Lx", "self._ex = idft_matrix(np.arange(nx + 1), self.jx, self.Px) / self.Ly / 2"),
    ('tbc.py', "padx, pady = cav.pad, cav.pad_y", "padx, pady = cav.pad, 2 * cav.pad_y"),
    ('tbc.py', "self._fy[kind] = phi_matrix(kind, ky, self.jy, b, pady)", "self._fy[kind] = phi_matrix(kind, ky, self.jy, b, padx)"),
    ('tbc.py', "self.Lx, self.Ly = padx * a, pady * b", "self.Lx, self.Ly = padx * a, padx * b"),
    ('tbc.py', "R = np.sqrt(2.0) * max(a, b)", "R = 1.3 * max(a, b)"),
    ('aperture.py', "wc[..., :, 1:] += self.ny[None, 1:] * e1", "wc[..., :, 1:] -= self.ny[None, 1:] * e1"),
    ('aperture.py', "y1 = (-1.0 + p.tau1) * e1", "y1 = (1.0 + p.tau1) * e1"),
    ('aperture.py', "y1[..., 1:, :] += (self.mx[1:, None] * h + p.vs1[1:, :]) * e3", "y1[..., 1:, :] += (self.mx[1:, None] * h - p.vs1[1:, :]) * e3"),
    ('aperture.py', "+ (self.ny[None, 1:] * h) * e2[..., :, 1:] + (-1.0 + p.tau3) * e3", "- (self.ny[None, 1:] * h) * e2[..., :, 1:] + (-1.0 + p.tau3) * e3"),
    ('aperture.py', "k2 = 2.0 * cav.kappa0 ** 2\n        h = cav.h\n        U1", "k2 = -2.0 * cav.kappa0 ** 2\n        h = cav.h\n        U1"),
    ('aperture.py', "(k2 * U2 + 2.0 * self.mx[1:, None] * W[1:, :])", "(k2 * U2 - 2.0 * self.mx[1:, None] * W[1:, :])"),
    ('aperture.py', "A[j1, i3] += (m3 * np.pi / cav.a * h + p.vs1[m3, q3 - 1]).ravel()", "A[j1, i3] += (m3 * np.pi / cav.a * h - p.vs1[m3, q3 - 1]).ravel()"),
    ('aperture.py', "A[i3, j2] += (q3 * np.pi / cav.b * h).ravel()", "A[i3, j2] += (q3 * np.pi / cav.a * h).ravel()"),
    ('aperture.py', "B21 = (s2 * 2.0 * mx[1:, None])[:, :, None, None] * \\\n            I3[1:, :, :, 1:]", "B21 = (s2 * 2.0 * mx[1:, None])[:, :, None, None] * \\\n            -I3[1:, :, :, 1:]"),
    ('tbc.py', "cy = nn + 1 if kind[1] == 'c' else nn", "cy = nn + 1"),
    ('field.py', "c1[1:, :] += prof.Q1[1:, :, j] * e3", "c1[1:, :] -= prof.Q1[1:, :, j] * e3"),
    ('field.py', "f2 = sinx @ c2 @ cosy.T", "f2 = sinx @ c2 @ cosy[::-1].T"),
    ('field.py', "siny = np.sin(np.pi * np.outer(py[1:-1], np.arange(1, N + 1)) / cav.ny)", "siny = np.sin(np.pi * np.outer(py[1:-1], np.arange(0, N)) / cav.ny)"),
    ('khat.py', "ez = np.exp(1j * kappa0 * r) * wt", "ez = np.exp(-1j * kappa0 * r) * wt"),
    ('khat.py', "out[idx] = 0.5 * (vals @ ez)", "out[idx] = 1.0 * (vals @ ez)"),
    ('khat.py', "vals = j0(2.0 * np.pi * flat[idx, None] * r[None, :])", "vals = j0(np.pi * flat[idx, None] * r[None, :])"),
    ('zsystem.py', "diag += 1.0          # Neumann: E_{3,0} = E_{3,1}", "diag += 0.0"),
    ('zsystem.py', "ab[1, 0] = s - 1.0                       # E_{3,0} = E_{3,1}", "ab[1, 0] = s - 2.0"),
    ('zsystem.py', "coef = mu * cav.h * (1.0 - cav.layers[up].eps / cav.layers[lo].eps)", "coef = mu * cav.h * (1.0 - cav.layers[lo].eps / cav.layers[up].eps)"),
    ('geometry.py', "k2 = self.kappa0 ** 2 * self.layers[layer_index].eps", "k2 = self.kappa0 ** 2"),
    ('geometry.py', "return (m * np.pi / self.a) ** 2 + (n * np.pi / self.b) ** 2", "return (m * np.pi / self.a) ** 2 + (n * np.pi / self.a) ** 2"),
    ('tbc.py', "rho = np.sqrt((ux[:, None] / self.Lx) ** 2 + (uy[None, :] / self.Ly) ** 2)", "rho = np.sqrt((ux[:, None] / self.Ly) ** 2 + (uy[None, :] / self.Lx) ** 2)"),
    ('tbc.py', "self._ey = idft_matrix(np.arange(ny + 1), self.jy, self.Py) / self.Ly", "self._ey = idft_matrix(np.arange(ny + 1), self.jy, self.Py) / self.Lx"),
    ('tbc.py', "h = P // 2 - 1", "h = P // 2 - 3"),
    ('tbc.py', "em = _E(2 * js - pad * ks, a, pad)", "em = _E(2 * js - pad * ks + 1, a, pad)"),
    ('excitation.py', "ph_hat = np.array([-sf, cf, 0.0])", "ph_hat = np.array([sf, -cf, 0.0])"),
    ('excitation.py', "sx = trap_matrix('s', np.arange(1, M + 1), cav.nx, cav.a) @ ex", "sx = trap_matrix('s', np.arange(0, M), cav.nx, cav.a) @ ex"),
    ('excitation.py', "y = np.arange(cav.ny + 1) * cav.b / cav.ny", "y = np.arange(cav.ny + 1) * cav.a / cav.ny"),
    ('aperture.py', "wc[..., 1:, :] -= self.mx[1:, None] * e2", "wc[..., 1:, :] += self.mx[1:, None] * e2"),
    ('aperture.py', "self.ny = np.arange(0, N + 1) * np.pi / cav.b", "self.ny = np.arange(0, N + 1) * np.pi / cav.a"),
    ('aperture.py', "y2 = (-1.0 + p.tau2) * e2", "y2 = (-1.0 + p.tau1[:p.tau2.shape[0], :p.tau2.shape[1]]) * e2"),
    ('zsystem.py', "rhs[-1, 0] = -1.0", "rhs[-1, 0] = 1.0"),
    ('field.py', "f1 = cosx @ c1 @ siny.T", "f1 = 0.5 * cosx @ c1 @ siny.T"),
    ('field.py', "f3 = sinx @ c3 @ siny.T", "f3 = -(sinx @ c3 @ siny.T)"),
    ('rcs.py', "return np.array([-I2, I1, 0.0 + 0j])", "return np.array([I2, I1, 0.0 + 0j])"),
    ('khat.py', "omega = 2.0 * np.pi * flat + abs(kappa0)", "omega = 0.2 * np.pi * flat + abs(kappa0)"),
    ('field.py', "c2[:, 1:] += prof.Q2[:, 1:, j] * e3", "c2[:, 1:] -= prof.Q2[:, 1:, j] * e3"),
    ('zsystem.py', "Q[1:nz] = sol[:, 1]", "Q[1:nz] = -sol[:, 1]"),
    ('zsystem.py', "_band_set(ab, U, ia, ia, -1.0)", "_band_set(ab, U, ia, ia, 1.0)"),
    ('zsystem.py', "self.vs2 = self.Q2[:, :, j]", "self.vs2 = -self.Q2[:, :, j]"),
    ('zsystem.py', "self.tau3 = self.P3[:, :, j]", "self.tau3 = self.P3[:, :, j - 1]"),
    ('zsystem.py', "d3 = p3[n - 1] if (layered and n >= 1) else None", "d3 = None"),
    ('aperture.py', "return ((m <= mm) & (n <= nn)).ravel()", "return ((m < mm) & (n <= nn)).ravel()"),
    ('excitation.py', "q = np.full(cav.M + 1, ab / 4.0)", "q = np.full(cav.M + 1, ab / 2.0)"),
    ('geometry.py', "res.append((top, li, li + 1))", "res.append((top - 1, li, li + 1))"),
    ('excitation.py', "p = np.cos(alpha) * th_hat + np.sin(alpha) * ph_hat", "p = np.sin(alpha) * th_hat + np.cos(alpha) * ph_hat"),
    ('khat.py', "tail = np.sqrt(2.0 / np.pi) / cb * (cos_part + sin_part / 8.0)", "tail = np.sqrt(2.0 / np.pi) / cb * (cos_part - sin_part / 8.0)"),
    ('khat.py', "pp, pm = k / cb + 1.0, k / cb - 1.0", "pp, pm = k / cb - 1.0, k / cb + 1.0"),
    ('khat.py', "out[big] = 0.5 * (inf - tail)", "out[big] = 0.5 * (inf + tail)"),
    ('aperture.py', "y2[..., :, 1:] += (self.ny[None, 1:] * h + p.vs2[:, 1:]) * e3", "y2[..., :, 1:] += (self.ny[None, 1:] * h) * e3"),
    ('tbc.py', "return (self._fx[kx].conj().T / self.Lx) @ V @ (self._fy[ky].conj() / self.Ly)", "return (self._fx[kx].T / self.Lx) @ V @ (self._fy[ky] / self.Ly)"),
    ('tbc.py', "            Xx = self._fx[kx].conj().T / self.Lx\n", "            Xx = self._fx[kx].conj().T\n"),
    ('tbc.py', "return (self._fx[kx].conj().T / self.Lx) @ V @ (self._fy[ky].conj() / self.Ly)", "return (self._fx[kx].conj().T / self.Lx) @ V @ (self._fy[ky].conj() / self.Lx)"),
    # the backscatter RCS, the kept block's remaining terms, the level map,
    # the trapezoid rule's far end and the x2 factors of the excitation
    ('rcs.py', "return 0.5 * (_ef(g - k, a) + _ef(g + k, a))", "return 0.5 * (_ef(g - k, a) - _ef(g + k, a))"),
    ('rcs.py', "return (_ef(g - k, a) - _ef(g + k, a)) / 2j", "return (_ef(g - k, a) - _ef(g + k, a)) / -2j"),
    ('rcs.py', "(1.0 - np.exp(-1j * safe * a)) / (1j * safe)", "(1.0 - np.exp(1j * safe * a)) / (1j * safe)"),
    ('rcs.py', "g1, g2 = cav.kappa0 * xh[0], cav.kappa0 * xh[1]", "g1, g2 = cav.kappa0 * xh[1], cav.kappa0 * xh[0]"),
    ('rcs.py', "e = np.array([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)])", "e = np.array([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), np.sin(theta)])"),
    ('rcs.py', "e = np.array([-np.sin(phi), np.cos(phi), 0.0])", "e = np.array([np.sin(phi), np.cos(phi), 0.0])"),
    ('rcs.py', "return cav.kappa0 ** 2 / np.pi * abs(v) ** 2", "return cav.kappa0 ** 2 / (4 * np.pi) * abs(v) ** 2"),
    ('rcs.py', "S1y = sin_int(np.arange(1, N + 1), g2, cav.b)", "S1y = sin_int(np.arange(1, N + 1), g2, cav.a)"),
    ('rcs.py', "I2 = S2x @ e2 @ C2y", "I2 = S2x @ e2 @ C2y.conj()"),
    ('aperture.py', "B12 = (s1 * 2.0 * ny[None, 1:])[:, :, None, None] * \\\n            I3[:, 1:, 1:, :]", "B12 = -(s1 * 2.0 * ny[None, 1:])[:, :, None, None] * \\\n            I3[:, 1:, 1:, :]"),
    ('aperture.py', "B22 -= (s2 * 2.0 * mx[1:, None])[:, :, None, None] * \\\n            I3[1:, :, 1:, :]", "B22 += (s2 * 2.0 * mx[1:, None])[:, :, None, None] * \\\n            I3[1:, :, 1:, :]"),
    ('aperture.py', "A[i2, i2] += (-1.0 + p.tau2[m2 - 1, q2]).ravel()", "A[i2, i2] += (1.0 + p.tau2[m2 - 1, q2]).ravel()"),
    ('aperture.py', "s2 = (h / self.cn[:nn + 1])[None, :]", "s2 = (h / self.cn[:nn + 1])[None, :] * 0.5"),
    ('geometry.py', "out[bot + 1:top] = li", "out[bot:top] = li"),
    ('tbc.py', "w[-1] *= 0.5", "w[-1] *= 1.0"),
    ('tbc.py', "arg = np.pi * np.outer(ms, p) / n_int", "arg = np.pi * np.outer(ms, p) / (n_int + 1)"),
    ('excitation.py', "cy = trap_matrix('c', np.arange(0, N + 1), cav.ny, cav.b) @ ey", "cy = trap_matrix('c', np.arange(0, N + 1), cav.ny, cav.b) @ ey.conj()"),
    ('excitation.py', "ey = np.exp(1j * a2 * y)", "ey = np.exp(1j * a1 * y)"),
]

KNOWN_SURVIVORS = {
    "h = P // 2 - 1",
}


# (original text, mutated text) in the block GMRES host numerics, checked
# against tests/test_block_host.py
HOST_HEADER = "paper_2008_01966_gb300/csrc/bgmres_host.h"
HOST_MUTATIONS = [
    ("const cd jpq = s * ph, jqp = -s * std::conj(ph);", "const cd jpq = s * ph, jqp = s * std::conj(ph);"),
    ("const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));", "const double t = (tau >= 0 ? -1.0 : 1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));"),
    ("for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * std::conj(L[(size_t)j * n + k]);", "for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];"),
    ("if (!(d > 1e-10 * dmax)) return false;", "if (!(d > 1e-20 * dmax)) return false;"),
    ("cond = std::sqrt(gf) * lf;", "cond = std::sqrt(gf * lf);"),
    ("T[(size_t)i * BG_MAX + j] = std::conj(Li[(size_t)j * n + i]);  // (L^{-1})^H", "T[(size_t)i * BG_MAX + j] = Li[(size_t)j * n + i];"),
    ("const double fl = lmax * 1e-12;", "const double fl = lmax * 1e-2;"),
    ("S[(size_t)c * n + i] = sl * std::conj(U[(size_t)i * n + c]);", "S[(size_t)c * n + i] = sl * U[(size_t)i * n + c];"),
    ("u[0] += ph * alpha;", "u[0] -= ph * alpha;"),
    ("for (int t = cols; t < rows; ++t) s += std::norm(g[(size_t)t * r + j]);", "for (int t = cols + 1; t < rows; ++t) s += std::norm(g[(size_t)t * r + j]);"),
    ("for (int k = i + 1; k < cols; ++k) s -= R[k][i] * Y[(size_t)k * BG_MAX + j];", "for (int k = i + 1; k < cols; ++k) s += R[k][i] * Y[(size_t)k * BG_MAX + j];"),
    ("for (int p = cols - (int)cix; p < cols; ++p) {", "for (int p = cols - (int)cix + 1; p < cols; ++p) {"),
    ("Y[(size_t)i * BG_MAX + j] = std::abs(d) > 0 ? s / d : cd(0, 0);", "Y[(size_t)i * BG_MAX + j] = s / d;"),
    ("o[(size_t)i * n + j] += a * S[(size_t)k * n + j];", "o[(size_t)i * n + j] += a * S[(size_t)j * n + k];"),
]


def run_host(a, b):
    tmp = tempfile.mkdtemp(prefix="host_mutant_")
    try:
        os.makedirs(os.path.join(tmp, os.path.dirname(HOST_HEADER)))
        shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(tmp, "tests"),
                        ignore=shutil.ignore_patterns("__pycache__"))
        src = open(os.path.join(ROOT, HOST_HEADER)).read()
        if src.count(a) != 1:
            return "site not found"
        open(os.path.join(tmp, HOST_HEADER), "w").write(src.replace(a, b))
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                            "tests/test_block_host.py"], cwd=tmp, capture_output=True, text=True,
                           timeout=600)
        return "caught" if r.returncode != 0 else "survived"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


def run_one(f, a, b):
    tmp = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(tmp, "oracle"),
                        ignore=shutil.ignore_patterns("__pycache__"))
        shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(tmp, "tests"),
                        ignore=shutil.ignore_patterns("__pycache__"))
        shutil.copy(os.path.join(ROOT, "workloads.py"), tmp)
        path = os.path.join(tmp, "oracle", f)
        src = open(path).read()
        if src.count(a) != 1:
            return "site not found"
        open(path, "w").write(src.replace(a, b))
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                            "tests/test_oracle_pins.py", "tests/test_khat_scheme.py"],
                           cwd=tmp, capture_output=True, text=True, timeout=900)
        return "caught" if r.returncode != 0 else "survived"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


def main():
    base = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                           "tests/test_oracle_pins.py", "tests/test_khat_scheme.py"],
                          cwd=ROOT, capture_output=True, text=True)
    if base.returncode != 0:
        print("the pins fail on the unmodified oracle; fix that first")
        return 2
    bad = 0
    for f, a, b in MUTATIONS:
        res = run_one(f, a, b)
        first = a.splitlines()[0]
        known = first in KNOWN_SURVIVORS
        print("%-9s %-14s %s%s" % (res, f, first[:70], "  (known)" if known and res == "survived" else ""),
              flush=True)
        if res != "caught" and not (known and res == "survived"):
            bad += 1
    for a, b in HOST_MUTATIONS:
        res = run_host(a, b)
        print("%-9s %-14s %s" % (res, "bgmres_host.h", a[:70]), flush=True)
        if res != "caught":
            bad += 1
    print("%d mutations, %d unexpected" % (len(MUTATIONS) + len(HOST_MUTATIONS), bad))
    return 1 if bad else 0


if __name__ == "__main__":
    sys.exit(main())
