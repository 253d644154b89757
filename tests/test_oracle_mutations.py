"""The oracle's pins against planted mistakes, CPU only.

Each mutant is a plausible slip in oracle/cue_oracle.c: a flipped sign, a
dropped neighbour, h for h^2, a transposed index, a swapped weight, a window
wall decided by the local index, a wrong constant of the generator, the field
stepped before the cones, a stop tested before the move, an off-by-one in a
wall, a binning or a graph step, the adjoint's decay, parameter scaling or
reverse-mode projections.  Each is planted alone in a copy of the oracle, which
is compiled and run against the pins that cover that part; every mutant must
make at least one pin fail.  (Clamping the cell index to N-1 instead of N-2 is
left out: it only ever gives the extra node weight 0, so it computes the same
values.)
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cue_oracle.c")

FIELD_CONE = ["tests/test_oracle_field.py", "tests/test_oracle_cone.py"]
SNR = ["tests/test_oracle_snr.py"]
GRAPH = ["tests/test_oracle_graph.py"]
ADJ = ["tests/test_oracle_adjoint.py"]

MUTANTS = [
    ("flux sign of one neighbour", "if (i > 0)      flux += C[c - sx] - ci;", "if (i > 0)      flux += ci - C[c - sx];",
     FIELD_CONE),
    ("dropped -y neighbour", "if (j > 0)      flux += C[c - sy] - ci;", "", FIELD_CONE),
    ("dropped -z neighbour", "if (k > 0)      flux += C[c - sz] - ci;", "", FIELD_CONE),
    ("h instead of h^2", "g->D * g->dt / (g->h * g->h);\n    const double decay = g->lambda * g->dt;\n    const int nx",
     "g->D * g->dt / (g->h);\n    const double decay = g->lambda * g->dt;\n    const int nx", FIELD_CONE),
    ("decay sign", "Cn[c] = ci + alpha * flux - decay * ci;", "Cn[c] = ci + alpha * flux + decay * ci;", FIELD_CONE),
    ("emission scaled by dt", "Cn[src_cell[s]] += src_emit[s];", "Cn[src_cell[s]] += src_emit[s] * g->dt;",
     FIELD_CONE),
    ("rate map not scaled by dt", "Cn[c] += g->dt * src_map[c];", "Cn[c] += src_map[c];", FIELD_CONE),
    ("central difference over h", "inv2h = 1.0 / (2.0 * g->h);\n    int nz = (g->dim",
     "inv2h = 1.0 / (g->h);\n    int nz = (g->dim", FIELD_CONE),
    ("interpolation weights swapped", "                double w = (di ? f[0] : 1.0 - f[0])",
     "                double w = (di ? 1.0 - f[0] : f[0])", FIELD_CONE),
    ("ghost node index", "node_value(g, C, clampi(i + 1, 0, g->nx - 1), j, k)",
     "node_value(g, C, clampi(i + 1, 0, g->nx - 2), j, k)", FIELD_CONE),
    ("noise word", "u2 = unit_open1(x[1]);", "u2 = unit_open1(x[2]);", FIELD_CONE),
    ("Weyl constant", "W0 = 0x9E3779B9u", "W0 = 0x9E3779B8u", FIELD_CONE),
    ("wall stop keeps the moved position", "active[a] = 0;          /* stays at p, d of this step */\n            continue;",
     "active[a] = 0; for (int c = 0; c < dim; ++c) pos[(size_t)c * n + a] = pn[c];\n            continue;", FIELD_CONE),
    ("source stop before the move", "d2 += (pn[c] - xs[c]) * (pn[c] - xs[c]);", "d2 += (p[c] - xs[c]) * (p[c] - xs[c]);",
     FIELD_CONE),
    ("source node decoded transposed", "xs[1] = (double)((cell / g->nx) % g->ny) * g->h;",
     "xs[1] = (double)((cell / g->ny) % g->nx) * g->h;", FIELD_CONE),
    ("gradient threshold ignored", "if (gn2 > eps2) {", "if (gn2 > 0.0) {", FIELD_CONE),
    ("blend weights swapped", "v[c] = cp->w_prev * d[c] + cp->w_grad * ghat[c]",
     "v[c] = cp->w_prev * ghat[c] + cp->w_grad * d[c]", FIELD_CONE),
    ("field stepped before the cones",
     "        if (n > 0)\n            orc_cone_step(g, cp, C, step, n, pos, dir, active, src_cell, n_src);\n"
     "        orc_field_step(g, C, work, src_cell, src_emit, n_src, src_map);\n"
     "        memcpy(C, work, (size_t)nn * sizeof(double));",
     "        orc_field_step(g, C, work, src_cell, src_emit, n_src, src_map);\n"
     "        memcpy(C, work, (size_t)nn * sizeof(double));\n"
     "        if (n > 0)\n            orc_cone_step(g, cp, C, step, n, pos, dir, active, src_cell, n_src);", FIELD_CONE),
    ("step length doubled", "pn[c] = p[c] + cp->step_len * dn[c];", "pn[c] = p[c] + 2 * cp->step_len * dn[c];",
     FIELD_CONE),
    ("wall one node out", "double hi = (extent(g, c) - 1) * g->h;", "double hi = extent(g, c) * g->h;", FIELD_CONE),
    ("Box-Muller cos and sin swapped", "xi[0] = r * cos(two_pi * u2);\n    xi[1] = r * sin(two_pi * u2);",
     "xi[0] = r * sin(two_pi * u2);\n    xi[1] = r * cos(two_pi * u2);", FIELD_CONE),
    ("3D interpolation weight swapped",
     "if (g->dim == 3) w *= (dk ? f[2] : 1.0 - f[2]);",
     "if (g->dim == 3) w *= (dk ? 1.0 - f[2] : f[2]);", FIELD_CONE),
    ("z ghost node index", "clampi(k + 1, 0, nz - 1)) -", "clampi(k + 1, 0, nz - 2)) -", FIELD_CONE),
    ("Philox with 9 rounds", "round < 10", "round < 9", FIELD_CONE),
    ("Philox multiplier", "M1 = 0xCD9E8D57u", "M1 = 0xCD9E8D56u", FIELD_CONE),
    ("Philox round key word", "uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi1 ^ c1 ^ k1;", FIELD_CONE),
    ("uniform (0,1] offset", "((double)(x >> 8) + 1.0)", "((double)(x >> 8) + 0.5)", FIELD_CONE),
    ("3D noise words swapped",
     "double u3 = unit_open0(x[2]), u4 = unit_open1(x[3]);",
     "double u3 = unit_open0(x[3]), u4 = unit_open1(x[2]);", FIELD_CONE),
    ("3D noise from the sine", "xi[2] = r2 * cos(two_pi * u4);", "xi[2] = r2 * sin(two_pi * u4);", FIELD_CONE),
    ("seed words swapped",
     "uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};",
     "uint32_t key[2] = {(uint32_t)(seed >> 32), (uint32_t)(seed & 0xFFFFFFFFu)};", FIELD_CONE),
    ("cone and step counter words swapped",
     "uint32_t ctr[4] = {axon, step, 0u, 0u};",
     "uint32_t ctr[4] = {step, axon, 0u, 0u};", FIELD_CONE),
    ("stop radius exclusive",
     "if (d2 <= r2) { active[a] = 0; break; }",
     "if (d2 < r2) { active[a] = 0; break; }", FIELD_CONE),
    ("wall clamp to the far wall", "pn[c] = pn[c] < 0.0 ? 0.0 : hi;", "pn[c] = pn[c] < 0.0 ? hi : 0.0;", FIELD_CONE),
    ("wall test inclusive", "if (pn[c] < 0.0 || pn[c] > hi) {", "if (pn[c] < 0.0 || pn[c] >= hi) {", FIELD_CONE),
    ("source node z decoded with nx*nx",
     "xs[2] = (dim == 3) ? (double)(cell / ((int64_t)g->nx * g->ny)) * g->h : 0.0;",
     "xs[2] = (dim == 3) ? (double)(cell / ((int64_t)g->nx * g->nx)) * g->h : 0.0;", FIELD_CONE),
    ("noise weighted by w_grad",
     "+ cp->w_noise * xi[c];\n                vn2",
     "+ cp->w_grad * xi[c];\n                vn2", FIELD_CONE),
    ("zero-blend fallback always taken",
     "if (vn2 > 1e-30) {\n                double inv",
     "if (vn2 > 1e30) {\n                double inv", FIELD_CONE),
    ("decay quadratic",
     "Cn[c] = ci + alpha * flux - decay * ci;",
     "Cn[c] = ci + alpha * flux - decay * ci * ci;", FIELD_CONE),
    ("window wall by local index", "if (gi > 0)      flux += Wp[c - sx] - ci;",
     "if (i > 0)      flux += Wp[c - sx] - ci;", FIELD_CONE),
    ("window top wall one row early", "if (gj < ny - 1) flux += Wp[c + sy] - ci;",
     "if (gj < ny - 2) flux += Wp[c + sy] - ci;", FIELD_CONE),
    ("window decay sign", "out[i + (int64_t)wx * (j + (int64_t)wy * k)] = ci + alpha * flux - decay * ci;",
     "out[i + (int64_t)wx * (j + (int64_t)wy * k)] = ci + alpha * flux + decay * ci;", FIELD_CONE),
    ("window source decoded transposed", "gj = (cell / nx) % ny, gk = cell / (nx * ny);",
     "gj = (cell / ny) % nx, gk = cell / (nx * ny);", FIELD_CONE),
    ("SNR turn direction", "(snr + xi[0] > 0.0) ? -cp->snr_turn : cp->snr_turn",
     "(snr + xi[0] > 0.0) ? cp->snr_turn : -cp->snr_turn", SNR),
    ("SNR window without its upper edge", "if (Cp >= cp->snr_cmin && Cp <= cp->snr_cmax) {",
     "if (Cp >= cp->snr_cmin) {", SNR),
    ("SNR sample weights swapped", "(dj ? f[1] : 1.0 - f[1]);\n            v += w",
     "(dj ? 1.0 - f[1] : f[1]);\n            v += w", SNR),
    ("SNR concentration exponent", "sqrt(gamma / (onep * onep * onep))", "sqrt(gamma / (onep * onep))", SNR),
    ("SNR rotation not a rotation", "r1 = d[0] * sn + d[1] * cs;", "r1 = -d[0] * sn + d[1] * cs;", SNR),
    ("SNR angle sign",
     "double sin_rel = (d[1] * gr[0] - d[0] * gr[1]) / gn;",
     "double sin_rel = (d[0] * gr[1] - d[1] * gr[0]) / gn;", SNR),
    ("SNR gamma inverted", "double gamma = Cp / cp->snr_kd;", "double gamma = cp->snr_kd / Cp;", SNR),
    ("SNR cone width ignored", "double mu = cp->snr_width * gn / Cp;", "double mu = gn / Cp;", SNR),
    ("SNR decision on the second draw", "(snr + xi[0] > 0.0)", "(snr + xi[1] > 0.0)", SNR),
    ("SNR window without its lower edge",
     "if (Cp >= cp->snr_cmin && Cp <= cp->snr_cmax) {",
     "if (Cp <= cp->snr_cmax) {", SNR),
    ("connection at the exact radius", "if (d2 < r2) {", "if (d2 <= r2) {", GRAPH),
    ("adjacency list keeps duplicates",
     "if (k == 0 || e[k].s != e[k - 1].s || e[k].d != e[k - 1].d) e[m++] = e[k];", "e[m++] = e[k];", GRAPH),
    ("BFS level step", "level[u] = level[v] + 1;", "level[u] = level[v] + 2;", GRAPH),
    ("cell end one short", "cell_end[pr[j].cell] = j + 1;", "cell_end[pr[j].cell] = j;", GRAPH),
    ("cone connects to its own neuron", "if (owner[a] == j) continue;", "", GRAPH),
    ("stopped cones connect", "if (active && !active[a]) continue;", "", GRAPH),
    ("edge source is the cone id", "src[count] = owner[a];", "src[count] = a;", GRAPH),
    ("ids within a cell in reverse",
     "return (x->id > y->id) - (x->id < y->id);",
     "return (x->id < y->id) - (x->id > y->id);", GRAPH),
    ("traversal by a stack", "int v = q[head++];", "int v = q[--tail];", GRAPH),
    ("row offsets shifted", "row[e[k].s + 1]++;", "row[e[k].s]++;", GRAPH),
    ("cell start one late",
     "if (j == 0 || pr[j].cell != pr[j - 1].cell) cell_start[pr[j].cell] = j;",
     "if (j == 0 || pr[j].cell != pr[j - 1].cell) cell_start[pr[j].cell] = j + 1;", GRAPH),
    ("adjoint decay sign", "mu2[c] = mu[c] + alpha * mu2[c] - decay * mu[c];",
     "mu2[c] = mu[c] + alpha * mu2[c] + decay * mu[c];", ADJ),
    ("dL/dlambda sign", "*glam -= g->dt * sL;", "*glam += g->dt * sL;", ADJ),
    ("dL/de scaled by dt", "gsrc[k] += mu[src_cell[k]];", "gsrc[k] += g->dt * mu[src_cell[k]];", ADJ),
    ("dL/dM not scaled by dt", "gmap[c] += g->dt * mu[c];", "gmap[c] += mu[c];", ADJ),
    ("loss adjoint without 1/n", "pbar[(size_t)k * n + a] = 2.0 * e / n;", "pbar[(size_t)k * n + a] = 2.0 * e;", ADJ),
    ("weight derivative without its sign", "dw[nc][1] = wx * sy * wz / g->h;", "dw[nc][1] = wx * wz / g->h;", ADJ),
    ("clamped move passes the adjoint", "qbar[k] = (q < 0.0 || q > hi) ? 0.0 : pbar[k];", "qbar[k] = pbar[k];", ADJ),
    ("normalisation adjoint without its projection",
     "vbar[k] = (dnbar[k] - dn[k] * dot) / vn;",
     "vbar[k] = dnbar[k] / vn;", ADJ),
    ("gradient normalisation adjoint without its projection",
     "gbar[k] = (cp->w_grad * vbar[k] - ghat[k] * dot) / gnorm;",
     "gbar[k] = (cp->w_grad * vbar[k]) / gnorm;", ADJ),
    ("sample position adjoint sign",
     "pbar_out[m] += gbar[k] * dw[c][m] * gn[c][k];",
     "pbar_out[m] -= gbar[k] * dw[c][m] * gn[c][k];", ADJ),
    ("field sample adjoint sign", "g->ny * ip[2])] += coef;", "g->ny * ip[2])] -= coef;", ADJ),
    ("step length dropped from the adjoint",
     "dnbar[k] = dbar[k] + cp->step_len * qbar[k];",
     "dnbar[k] = dbar[k] + qbar[k];", ADJ),
    ("dL/dD without 1/h^2", "*gD += alpha_dD * sD;", "*gD += g->dt * sD;", ADJ),
    ("adjoint Laplacian without -y", "if (j > 0) s += x[c - sy] - xi;", "", ADJ),
    ("direction adjoint without w_prev", "dbar_out[k] = cp->w_prev * vbar[k];", "dbar_out[k] = vbar[k];", ADJ),
    ("weight derivative along z dropped",
     "dw[nc][2] = (dim == 3) ? wx * wy * sz / g->h : 0.0;",
     "dw[nc][2] = 0.0;", ADJ),
]


def _run(mutant, src):
    name, old, new, pins = mutant
    d = tempfile.mkdtemp(prefix="orc_mut_")
    try:
        shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"),
                        ignore=shutil.ignore_patterns("_build", "__pycache__"))
        shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(d, "tests"),
                        ignore=shutil.ignore_patterns("__pycache__"))
        shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
        with open(os.path.join(d, "oracle", "cue_oracle.c"), "w") as f:
            f.write(src.replace(old, new, 1))
        env = dict(os.environ, OMP_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                            *pins], cwd=d, capture_output=True, text=True, timeout=900, env=env)
        # exit code 1: the pins ran and at least one failed (2+: the copy did not even build or collect)
        return name, r.returncode, r.stdout[-400:]
    finally:
        shutil.rmtree(d, ignore_errors=True)


def test_every_planted_mistake_fails_a_pin():
    with open(SRC) as f:
        src = f.read()
    for name, old, _, _ in MUTANTS:
        assert src.count(old) == 1, f"mutant '{name}' no longer matches the oracle source"
    workers = max(1, min(len(MUTANTS), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as pool:
        results = list(pool.map(lambda m: _run(m, src), MUTANTS))
    survived = [(name, rc, tail) for name, rc, tail in results if rc != 1]
    assert not survived, survived
