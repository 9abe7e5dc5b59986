"""Mutation check of the oracle's pins (CPU only, not collected by pytest).

Plants one plausible mistake at a time (a dropped term, a wrong sign, index
or bound, transposed operands) in a scratch copy of oracle/cch_oracle.c,
rebuilds it there and runs the oracle pin tests against it; a mistake the
pins do not catch is reported as SURVIVED.  The repository itself is never
modified.

    python tests/mutation_check.py            # every mutant, 6 at a time
    python tests/mutation_check.py 3 17 40    # selected mutants
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
M = [
    ("ps_dist clamps t<=0 to the wrong end", "if (t <= 0.0) { t = 0.0; q = a; }", "if (t <= 0.0) { t = 0.0; q = b; }"),
    ("pt_dist inside test bound", "u + v <= 1.0) return", "u + v <= 1.5) return"),
    ("pt_closest weights swapped", "wt[0] = (1.0 - u) - v; wt[1] = u; wt[2] = v;", "wt[0] = (1.0 - u) - v; wt[1] = v; wt[2] = u;"),
    ("ss_dist interior s sign", "double s = (B * F - C * E) / den", "double s = (B * F + C * E) / den"),
    ("ss_dist endpoint parameter", "dd = ps_dist(b, c, d, &tt); if (dd < best) { best = dd; bs = 1.0;", "dd = ps_dist(b, c, d, &tt); if (dd < best) { best = dd; bs = 0.0;"),
    ("ss_dist drops an endpoint case", "  dd = ps_dist(d, a, b, &tt); if (dd < best) { best = dd; bs = tt; bt = 1.0; }\n", ""),
    ("cross3 y component sign", "a.z * b.x - a.x * b.z", "a.x * b.z - a.z * b.x"),
    ("box_near boundary", "if (b->lo[k] - a->hi[k] > D) return 0;", "if (b->lo[k] - a->hi[k] >= D) return 0;"),
    ("all_static checks one vertex", "if (!s->is_static[v[i]]) return 0;", "if (!s->is_static[v[0]]) return 0;"),
    ("VT adjacency exclusion dropped (all-pairs)", "        if (a == tv[0] || a == tv[1] || a == tv[2]) continue;\n        int32_t v4[4] = {a, tv[0], tv[1], tv[2]};\n        if (all_static(s, v4, 4)) continue;\n        if (box_near(&vb[qi], &tb[tr], D)) kv_push(out, mkkey(ORC_VT, a, tr));\n      }\n    }\n  } else {", "        if (a == tv[0] || a == tv[1]) continue;\n        int32_t v4[4] = {a, tv[0], tv[1], tv[2]};\n        if (all_static(s, v4, 4)) continue;\n        if (box_near(&vb[qi], &tb[tr], D)) kv_push(out, mkkey(ORC_VT, a, tr));\n      }\n    }\n  } else {"),
    ("VV point pair counted twice", "if (s->is_point[b] && b < a) continue;", "if (s->is_point[b] && b < a && 0) continue;"),
    ("window slack zero", "slack = 1e-9 * (1.0 + M) + 1e-9 * D;", "slack = 0.0;"),
    ("window misses the widest box", "double from = vb[qi].lo[ax] - D - W - slack", "double from = vb[qi].lo[ax] - D - slack"),
    ("orient3d exact sign of one term", "ex_det3(&e, 1.0, a, b, d); ex_det3(&e, -1.0, a, b, c);", "ex_det3(&e, 1.0, a, b, d); ex_det3(&e, 1.0, a, b, c);"),
    ("orient3d filter bound too small", "double bound = 5e-15 * perm;", "double bound = 0.0 * perm;"),
    ("splitmix constant", "0xbf58476d1ce4e5b9ULL", "0xbf58476d1ce4e5b8ULL"),
    ("volume c sign", "*c0 = dx / dr - 1.0;", "*c0 = dx / dr + 1.0;"),
    ("volume gradient of p2 transposed", "g[2] = div3(cross3(c3, c1), dr);", "g[2] = div3(cross3(c1, c3), dr);"),
    ("volume reference shift sign", "r[i] = add3(p[i], scl3(sgn[i] * h, n));", "r[i] = add3(p[i], scl3(-sgn[i] * h, n));"),
    ("gap c drops -1", "*c0 = d / delta - 1.0;", "*c0 = d / delta;"),
    ("VT side flipped", "double side = dot3(nh, sub3(p[0], p[1])) < 0.0 ? -1.0 : 1.0;", "double side = dot3(nh, sub3(p[0], p[1])) < 0.0 ? 1.0 : -1.0;"),
    ("VT reference moves vertex with triangle", "static const double sg[4] = {1.0, -1.0, -1.0, -1.0};", "static const double sg[4] = {1.0, 1.0, -1.0, -1.0};"),
    ("EE gap weights swapped", "double w[4] = {1.0 - s, s, -(1.0 - t), -t};", "double w[4] = {s, 1.0 - s, -(1.0 - t), -t};"),
    ("EE parallel threshold", "nn < 1e-12 * (", "nn < 1e-40 * ("),
    ("VV drops one radius", "double R = (ra + rb) + delta;", "double R = ra + delta;"),
    ("PGS update sign", "double sc = im[c->v[k]] * dl;", "double sc = -im[c->v[k]] * dl;"),
    ("PGS residual operands transposed", "w = w + dot3(c->g[k], sub3(ld3(y, c->v[k]), ld3(x, c->v[k])));", "w = w + dot3(c->g[k], sub3(ld3(x, c->v[k]), ld3(y, c->v[k])));"),
    ("PGS no projection", "  double tl = c->lambda - w / c->den;\n  double ln = tl > 0.0 ? tl : 0.0;\n  double dl = ln - c->lambda;\n  c->lambda = ln;\n  if (dl == 0.0) return;\n  for (int k", "  double tl = c->lambda - w / c->den;\n  double ln = tl;\n  double dl = ln - c->lambda;\n  c->lambda = ln;\n  if (dl == 0.0) return;\n  for (int k"),
    ("edge constraint sign", "double w = sigma - dot3(c->g[0], sub3(ld3(y, c->v[0]), ld3(y, c->v[1])));", "double w = sigma + dot3(c->g[0], sub3(ld3(y, c->v[0]), ld3(y, c->v[1])));"),
    ("edge update of j sign", "st3(y, c->v[1], add3(ld3(y, c->v[1]), scl3(sj, c->g[0])));", "st3(y, c->v[1], sub3(ld3(y, c->v[1]), scl3(sj, c->g[0])));"),
    ("edge gradient misses 1/L0", "c->g[0] = div3(div3(d0, L0), L0);", "c->g[0] = div3(d0, L0);"),
    ("edge den misses m_j", "c->den = (t->inv_mass[i] + t->inv_mass[j]) * dot3(c->g[0], c->g[0]);", "c->den = t->inv_mass[i] * dot3(c->g[0], c->g[0]);"),
    ("contact den misses a vertex", "for (int k = 0; k < c->nv; k++) c->den = c->den + t->inv_mass[c->v[k]] * dot3(c->g[k], c->g[k]);", "for (int k = 1; k < c->nv; k++) c->den = c->den + t->inv_mass[c->v[k]] * dot3(c->g[k], c->g[k]);"),
    ("contact activation boundary", "if (!(P->d[i] < prm->delta)) continue;", "if (!(P->d[i] < 1.5 * prm->delta)) continue;"),
    ("Jacobi without per-constraint relaxation", "return omega / (double)(m > 0 ? m : 1);", "return omega;"),
    ("Jacobi lambda advance", "cc[i].lambda = cc[i].lambda + sc[i];", "cc[i].lambda = cc[i].lambda + 2.0 * sc[i];"),
    ("edges before contacts", "    for (int64_t i = 0; i < nc; i++) pgs_contact(&cc[i], x, y, t->inv_mass);\n    for (int64_t i = 0; i < ne; i++) pgs_edge(&ce[i], prm->sigma, y, t->inv_mass);", "    for (int64_t i = 0; i < ne; i++) pgs_edge(&ce[i], prm->sigma, y, t->inv_mass);\n    for (int64_t i = 0; i < nc; i++) pgs_contact(&cc[i], x, y, t->inv_mass);"),
    ("ascending priority", "return pa > pb ? -1 : pa < pb;", "return pa < pb ? -1 : pa > pb;"),
    ("colour classes swept in descending colour", "if (ca->colour != cb->colour) return ca->colour < cb->colour ? -1 : 1;", "if (ca->colour != cb->colour) return ca->colour > cb->colour ? -1 : 1;"),
    ("colouring conflicts through static vertices", "      if (movable[cs[i].v[k]]) mv[nm++] = cs[i].v[k];", "      mv[nm++] = cs[i].v[k];"),
    ("colouring ignores the last vertex's colours", "    for (int k = 0; k < nm; k++)\n      for (int32_t j = 0;", "    for (int k = 0; k + 1 < nm; k++)\n      for (int32_t j = 0;"),
    ("colouring without classes (priority order only)", "  qsort(cc, (size_t)nc, sizeof(cons), cmp_cons_colour);", "  qsort(cc, (size_t)nc, sizeof(cons), cmp_cons_prio_desc);"),
    ("contact multipliers kept (equivalent: rebuilt at 0)", "  for (int64_t i = 0; i < nc; i++) cc[i].lambda = 0.0;\n", ""),
    ("forward step uses gamma not gamma/2", "double q = (hg * bound) / nd;", "double q = (2.0 * hg * bound) / nd;"),
    ("CCD rule uses D_i", "double bound = ccd_rule ? (Di[v] == 0.0 ? 0.0 : Dcap) : Di[v];", "double bound = ccd_rule ? Di[v] : Di[v];"),
    ("CCD rule ignores the D_i floor", "double bound = ccd_rule ? (Di[v] == 0.0 ? 0.0 : Dcap) : Di[v];", "double bound = ccd_rule ? Dcap : Di[v];"),
    ("r update", "r[v] = r[v] * (1.0 - alpha[v]);", "r[v] = r[v] * alpha[v];"),
    ("D update halves the move", "D = nextafter(D - 2.0 * mmax, -INFINITY);", "D = nextafter(D - mmax, -INFINITY);"),
    ("D_i from the first vertex only", "if (P.d[i] < Di[v4[k]]) Di[v4[k]] = P.d[i];", "if (P.d[i] < Di[v4[0]]) Di[v4[0]] = P.d[i];"),
    ("refresh keeps far pairs", "if (d < D) { P.k[m] = P.k[i]; P.d[m] = d; m++; }", "if (d < 2.0 * D) { P.k[m] = P.k[i]; P.d[m] = d; m++; }"),
    ("search schedule", "if (D < prm->d_min) {", "if (D < 0.5 * prm->d_min) {"),
    ("no distance floor", "if (!(Di[v] >= ORC_D_FLOOR)) Di[v] = 0.0;", "if (0) Di[v] = 0.0;"),
    ("step_to returns x at a = 1", "  if (a == 1.0) return y;\n  if (a == 0.0) return x;\n  return add3", "  if (a == 1.0) return x;\n  if (a == 0.0) return x;\n  return add3"),
    ("non-finite y moves", "        a = 0.0; /* R2c: y not finite, the vertex does not move */", "        a = 1.0;"),
    ("CCD cubic drops a term", "c[1] = (det3(b[0], a[1], a[2]) + det3(a[0], b[1], a[2])) + det3(a[0], a[1], b[2]);", "c[1] = det3(b[0], a[1], a[2]) + det3(a[0], b[1], a[2]);"),
    ("CCD touch tolerance", "#define CCD_TOUCH 1e-9", "#define CCD_TOUCH 1e-3"),
    ("CCD clamp factor", "if (0.5 * toi < clampf[v4[k]]) clampf[v4[k]] = 0.5 * toi;", "if (0.9 * toi < clampf[v4[k]]) clampf[v4[k]] = 0.9 * toi;"),
    ("freeze keeps the tentative positions", "for (int64_t v = 0; v < n; v++) { alpha[v] = 0.0; st3(xn, v, ld3(x, v)); }", "for (int64_t v = 0; v < n; v++) { alpha[v] = 0.0; }"),
    ("VV CCD misses the radius", "double rr = dot3(r, r), RR = (R + CCD_TOUCH) * (R + CCD_TOUCH);", "double rr = dot3(r, r), RR = CCD_TOUCH * CCD_TOUCH;"),
    ("seg-tri: same side test ignores zero", "if (s1 != 0 && s1 == s2) return 0;", "if (s1 == s2) return 0;"),
    ("seg-tri: mixed signs accepted", "  if (pos && neg) return 0;\n  if (pos == 0 && neg == 0)", "  if (pos && neg && 0) return 0;\n  if (pos == 0 && neg == 0)"),
    ("intersections prune touching boxes", "if (!box_near(&eb[e], &tb[tr], 0.0)) continue;", "if (!box_near(&eb[e], &tb[tr], -1e-6)) continue;"),
    ("point-in-triangle open", "return !(pos && neg);", "return !(pos && neg) && pos + neg == 3;"),
    ("edge multipliers kept across steps", "  for (int64_t i = 0; i < ne; i++) ce[i].lambda = 0.0;\n", ""),
    ("collinear overlap test", "return (q.x >= fmin(a.x, b.x) && q.x <= fmax(a.x, b.x)", "return (q.x > fmin(a.x, b.x) && q.x < fmax(a.x, b.x)"),
]


def run(i):
    desc, old, new = M[i]
    d = tempfile.mkdtemp(prefix=f"mut{i}_")
    try:
        for sub in ("oracle", "tests", "paper_2211_04045_gb300"):
            shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                            ignore=shutil.ignore_patterns("_build", "__pycache__", "*.so", "*.o"))
        shutil.copy(os.path.join(ROOT, "bench.py"), d)  # the serving inputs' generator
        src = os.path.join(d, "oracle", "cch_oracle.c")
        s = open(src).read()
        if old not in s:
            return i, desc, "NOT APPLIED"
        open(src, "w").write(s.replace(old, new, 1))
        tests = sorted(os.path.join("tests", f) for f in os.listdir(os.path.join(d, "tests"))
                       if f.startswith("test_oracle_") or f in ("test_scene_inputs.py",))
        p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            "--deselect", "tests/test_oracle_regression.py::test_c_abi_defaults_are_table_2", *tests], cwd=d,
                           capture_output=True, text=True, timeout=1800)
        last = [l for l in p.stdout.splitlines() if l.strip()][-1:] or ["?"]
        if p.returncode == 0:
            return i, desc, "SURVIVED " + last[0]
        failed = [l for l in p.stdout.splitlines() if l.startswith("FAILED")][:1]
        return i, desc, "killed: " + (failed[0][7:90] if failed else last[0][:80])
    finally:
        shutil.rmtree(d, ignore_errors=True)


if __name__ == "__main__":
    with cf.ProcessPoolExecutor(6) as ex:
        which = [int(a) for a in sys.argv[1:]] or range(len(M))
        for i, desc, res in sorted(ex.map(run, which)):
            print(f"{i:2d} {desc:45s} {res}", flush=True)
