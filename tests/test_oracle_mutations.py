"""The oracle's pins catch planted mistakes.

Each case copies the oracle into a temporary directory, plants one plausible
mistake in oracle.c (a dropped term, a wrong exponent, sign, index or
rounding), builds it there and runs the pin suite against it: at least one pin
must fail.  Everything runs on the CPU; nothing here touches the GPU path.
"""

import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("alpha/2 -> alpha", "double w_den = pow(W, alpha / 2.0);", "double w_den = pow(W, alpha);"),
    ("median upper middle only", ": 0.5 * (sorted_rho[m2 / 2 - 1] + sorted_rho[m2 / 2]);",
     ": sorted_rho[m2 / 2];"),
    ("2 sigma^2 -> sigma^2", "exp(-d2 / (2.0 * (sigma * sigma) * r2i))", "exp(-d2 / ((sigma * sigma) * r2i))"),
    ("gamma/2 -> gamma", "double D = pow(d2, gamma / 2.0);", "double D = pow(d2, gamma);"),
    ("percentile ceil -> floor", "double cc = ceil(pos);", "double cc = floor(pos);"),
    (">= n_v -> > n_v", "if (k >= p->min_vox_count) p1[n1++]", "if (k > p->min_vox_count) p1[n1++]"),
    ("neighbour tie-break reversed",
     "if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;\n  return 0;\n}\n\nstatic int cmp_double",
     "if (x->idx != y->idx) return x->idx > y->idx ? -1 : 1;\n  return 0;\n}\n\nstatic int cmp_double"),
    ("leaf test <= cap -> < cap", "if (count <= o->cap || level", "if (count < o->cap || level"),
    ("density uses K not k_eff", "rho[a] = (double)keff /", "rho[a] = (double)p->k /"),
    ("Morton x/z bits swapped", "key |= (uint64_t)((qx >> b) & 1u) << (3 * b + 2);",
     "key |= (uint64_t)((qx >> b) & 1u) << (3 * b);"),
    ("median over P_1", "if (in2[a]) sorted_rho[m2++] = rho[a];", "if (in2[a]) m2++;"),
    ("W uses rho_i twice", "double W = rho[a] * rho[b] / wden_den;", "double W = rho[a] * rho[a] / wden_den;"),
    ("eps_k dropped", "double kern = 1.0 / (D + eps_k);", "double kern = 1.0 / (D);"),
    ("extent floor dropped", "if (H[a] < c->delta) H[a] = c->delta;", ""),
    ("r_K floor dropped", "r2[a] = (rk2 < delta2) ? delta2 : rk2;", "r2[a] = rk2;"),
    ("d/dsigma sign", "dS += t * d2 / (sigma * sigma * sigma * r2i);", "dS -= t * d2 / (sigma * sigma * sigma * r2i);"),
    ("sigmoid slope drops 1/T", "dm[i] = m * (1.0 - m) / T;", "dm[i] = m * (1.0 - m);"),
    ("Top-lambda floor", "double want = ceil((double)p->lambda * (double)m2);",
     "double want = floor((double)p->lambda * (double)m2);"),
    ("cube root 3 Newton steps", "for (int it = 0; it < 10; ++it) {", "for (int it = 0; it < 3; ++it) {"),
    ("threshold log -> log10", "(log(rk[t].f) >= (double)p->tau)", "(log10(rk[t].f) >= (double)p->tau)"),
    ("threshold >= -> >", "(log(rk[t].f) >= (double)p->tau)", "(log(rk[t].f) > (double)p->tau)"),
    ("threshold on F, not ln F", "(log(rk[t].f) >= (double)p->tau)", "(rk[t].f >= (double)p->tau)"),
    ("soft removal on F, not ln F (gradient kept consistent)",
     ("double z = (log(F[i]) - tau) / T;", "double dr_dF = -dm[i] / F[i];"),
     ("double z = (F[i] - tau) / T;", "double dr_dF = -dm[i];")),
    ("soft removal sign of tau", "double z = (log(F[i]) - tau) / T;", "double z = (log(F[i]) + tau) / T;"),
    ("Chamfer second term dropped", "if (cd) *cd = m + sb / (double)nb;", "if (cd) *cd = m;"),
    ("PSNR with M not M^2", "if (psnr) *psnr = 10.0 * log10(M2 / m);", "if (psnr) *psnr = 10.0 * log10(sqrt(M2) / m);"),
    ("MSE over the denoised cloud", "const double m = sa / (double)na;", "const double m = sb / (double)nb;"),
    ("baseline radius factor 6 -> 3", "const double R = 6.0 * (H[0] * H[1]", "const double R = 3.0 * (H[0] * H[1]"),
    ("baseline self not counted", "cnt += ((double)d2 <= R2);", "cnt += ((double)d2 <= R2) && j != i;"),
    ("baseline Eq. 8 with d^2", "keep[i] = F >= T / d;", "keep[i] = F >= T / (d * d);"),
    ("baseline centroid over N-1", "for (int c = 0; c < 3; ++c) theta[c] /= (double)n;",
     "for (int c = 0; c < 3; ++c) theta[c] /= (double)(n - 1);"),
    ("variant: voxel gate never switched off", "    if (!a1_on) {  /* the voxel gate is off", "    if (0) {  /* the voxel gate is off"),
    ("variant: score selection never switched off", "  if (!a3_on) {  /* no score selection", "  if (0) {  /* no score selection"),
    ("variant: rescoring ignored", "  if (p->rescore_p2) {", "  if (0) {"),
    ("cross-leaf: own cell only", "    for (int dx = -1; dx <= 1; ++dx)\n      for (int dy = -1; dy <= 1; ++dy)\n        for (int dz = -1; dz <= 1; ++dz) {",
     "    for (int dx = 0; dx <= 0; ++dx)\n      for (int dy = 0; dy <= 0; ++dy)\n        for (int dz = 0; dz <= 0; ++dz) {"),
    ("cross-leaf: score exponent alpha", "F += pow(W, alpha / 2.0) * exp(", "F += pow(W, alpha) * exp("),
    ("cross-leaf: eps_k dropped", "const double kern = 1.0 / (pow(d2, gamma / 2.0) + eps_k);",
     "const double kern = 1.0 / (pow(d2, gamma / 2.0));"),
    ("voxel origin shifted", "float d = coord(c, idx[t], a) - lo[a];", "float d = coord(c, idx[t], a) - lo[a] + h * 0.5f;"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    olds, news = (old, new) if isinstance(old, tuple) else ((old,), (new,))
    for o in olds:
        assert o in src, f"mutation site for '{name}' no longer exists"
    for sub in ("oracle", "tests", "synth", "paper_2512_10386_gb300"):
        shutil.copytree(os.path.join(ROOT, sub), tmp_path / sub,
                        ignore=shutil.ignore_patterns("*.so", "__pycache__", "_build"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path)
    for o, n in zip(olds, news):
        src = src.replace(o, n, 1)
    (tmp_path / "oracle" / "oracle.c").write_text(src)
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x",
                        "-p", "no:cacheprovider"], cwd=tmp_path, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"planted mistake '{name}' passed every pin:\n{r.stdout[-500:]}"
