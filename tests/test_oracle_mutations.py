"""The oracle's pins against planted mistakes, CPU only.

Each mutant is a plausible slip in oracle/cue_oracle.c — a flipped sign, a
dropped neighbour, h for h^2, a transposed index, a swapped weight, a wrong
constant of the generator, the field stepped before the cones, a stop tested
before the move, an off-by-one in a wall, a binning or a graph step, the
adjoint's decay or parameter scaling — planted in a copy of the oracle, which is
compiled and run against the pins that cover that part.  Every mutant must make
at least one pin fail.  (Clamping the cell index to N-1 instead of N-2 is left
out: it only ever gives the extra node weight 0, so it computes the same
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
    ("SNR turn direction", "(snr + xi[0] > 0.0) ? -cp->snr_turn : cp->snr_turn",
     "(snr + xi[0] > 0.0) ? cp->snr_turn : -cp->snr_turn", SNR),
    ("SNR window without its upper edge", "if (Cp >= cp->snr_cmin && Cp <= cp->snr_cmax) {",
     "if (Cp >= cp->snr_cmin) {", SNR),
    ("SNR sample weights swapped", "(dj ? f[1] : 1.0 - f[1]);\n            v += w",
     "(dj ? 1.0 - f[1] : f[1]);\n            v += w", SNR),
    ("SNR concentration exponent", "sqrt(gamma / (onep * onep * onep))", "sqrt(gamma / (onep * onep))", SNR),
    ("connection at the exact radius", "if (d2 < r2) {", "if (d2 <= r2) {", GRAPH),
    ("adjacency list keeps duplicates",
     "if (k == 0 || e[k].s != e[k - 1].s || e[k].d != e[k - 1].d) e[m++] = e[k];", "e[m++] = e[k];", GRAPH),
    ("BFS level step", "level[u] = level[v] + 1;", "level[u] = level[v] + 2;", GRAPH),
    ("cell end one short", "cell_end[pr[j].cell] = j + 1;", "cell_end[pr[j].cell] = j;", GRAPH),
    ("adjoint decay sign", "mu2[c] = mu[c] + alpha * mu2[c] - decay * mu[c];",
     "mu2[c] = mu[c] + alpha * mu2[c] + decay * mu[c];", ADJ),
    ("dL/dlambda sign", "*glam -= g->dt * sL;", "*glam += g->dt * sL;", ADJ),
    ("dL/de scaled by dt", "gsrc[k] += mu[src_cell[k]];", "gsrc[k] += g->dt * mu[src_cell[k]];", ADJ),
    ("dL/dM not scaled by dt", "gmap[c] += g->dt * mu[c];", "gmap[c] += mu[c];", ADJ),
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
