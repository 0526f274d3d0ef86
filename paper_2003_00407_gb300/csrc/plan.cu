// Host planning for libdgdft (no device code).
#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>

#include "plan.h"

namespace dgdft {

bool factor_line(int n, int& n1, int& n2) {
  static const int rad[] = {1, 2, 3, 4, 5, 6, 8};
  int best = 1 << 30;
  bool ok = false;
  for (int a : rad)
    for (int b : rad)
      if (a * b == n) {
        const int cost = std::max(a, b) * 16 - b;  // balanced, then larger second pass
        if (cost < best) { best = cost; n1 = a; n2 = b; ok = true; }
      }
  return ok;
}

static double min_image(double d, double L) { return d - L * std::nearbyint(d / L); }

static int nblk_rule(int n_eig) {
  const int g = std::max(4, (n_eig + 9) / 10);
  return 8 * ((n_eig + g + 7) / 8);
}

// Minimal cyclic run of region indices whose minimum-image displacement from
// the atom is within r_cut along one axis.  Returns false when there is none.
static bool axis_run(int r0, int nreg, int ndom, double h, double R, double rc, int& s, int& l,
                     std::vector<double>& disp, double& dmin) {
  const double L = ndom * h;
  // quick reject: the atom's image nearest to the region centre is too far
  const double centre = (r0 + 0.5 * (nreg - 1)) * h;
  if (nreg < ndom && std::fabs(min_image(R - centre, L)) > 0.5 * (nreg - 1) * h + rc) return false;
  std::vector<char> in(nreg);
  std::vector<double> dd(nreg);
  int cnt = 0;
  dmin = 1e300;
  for (int i = 0; i < nreg; i++) {
    const int g = ((r0 + i) % ndom + ndom) % ndom;
    dd[i] = min_image(g * h - R, L);
    in[i] = std::fabs(dd[i]) < rc;
    cnt += in[i];
    dmin = std::min(dmin, std::fabs(dd[i]));
  }
  if (cnt == 0) return false;
  if (cnt == nreg) {
    s = 0;
    l = nreg;
  } else {
    // longest cyclic gap of outside indices; the run starts right after it
    int best_len = -1, best_end = 0;
    for (int i = 0; i < nreg; i++) {
      if (in[i] || !in[(i - 1 + nreg) % nreg]) continue;  // i starts a gap
      int len = 0;
      while (!in[(i + len) % nreg]) len++;
      if (len > best_len) { best_len = len; best_end = (i + len) % nreg; }
    }
    s = best_end;
    l = nreg - best_len;
  }
  disp.resize(l);
  for (int i = 0; i < l; i++) disp[i] = dd[(s + i) % nreg];
  return true;
}

static void atom_boxes(const dgdft_problem* pr, const ElemDesc& d, const int r0[3], const int rn[3], int& begin,
                       int& count, int& ncol, Plan& P) {
  begin = int(P.boxes.size());
  count = 0;
  ncol = 0;
  const int npa = pr->n_proj_per_atom;
  for (int a = 0; a < pr->n_atoms; a++) {
    if (pr->atom_dom[a] != d.dom) continue;
    int s[3], l[3];
    std::vector<double> disp[3];
    double dmin[3];
    bool ok = true;
    for (int ax = 0; ax < 3 && ok; ax++)
      ok = axis_run(r0[ax], rn[ax], d.gn[ax], d.h[ax], pr->atom_pos[3 * a + ax], pr->r_cut, s[ax], l[ax], disp[ax],
                    dmin[ax]);
    if (!ok) continue;
    if (dmin[0] * dmin[0] + dmin[1] * dmin[1] + dmin[2] * dmin[2] >= pr->r_cut * pr->r_cut) continue;
    AtomBox b{};
    b.atom = a;
    for (int ax = 0; ax < 3; ax++) { b.s[ax] = s[ax]; b.l[ax] = l[ax]; }
    b.toff = int(P.dtab.size());
    for (int ax = 0; ax < 3; ax++) P.dtab.insert(P.dtab.end(), disp[ax].begin(), disp[ax].end());
    b.col = ncol;
    b.depth = pr->well_depth[a];
    b.wwidth = pr->well_width[a];
    const double sig = pr->proj_width ? pr->proj_width[a] : 1.0;
    b.pwidth = sig;
    b.ns = std::pow(M_PI * sig * sig, -0.75);
    b.np = std::sqrt(2.0) / sig * b.ns;
    for (int l2 = 0; l2 < 4; l2++) b.gamma[l2] = (l2 < npa) ? pr->proj_gamma[a * npa + l2] : 0.0;
    P.boxes.push_back(b);
    count++;
    ncol += npa;
  }
}

int build_plan(const dgdft_problem* pr, const dgdft_alb_params* prm, Plan& P, std::string& msg) {
  auto bad = [&](const std::string& m) { msg = m; return int(DGDFT_INVALID_ARG); };
  auto unsup = [&](const std::string& m) { msg = m; return int(DGDFT_UNSUPPORTED); };
  if (!pr || !prm) return bad("null problem or params");
  if (pr->n_dom < 1 || !pr->dom_n || !pr->dom_h || !pr->dom_voff) return bad("domains missing");
  if (pr->n_elem < 1 || !pr->elem_dom || !pr->elem_E0 || !pr->elem_En || !pr->elem_Qn) return bad("elements missing");
  if (!prm->n_eig || !prm->n_alb) return bad("n_eig / n_alb missing");
  if (!(pr->n_stencil == 1 || pr->n_stencil == 3 || pr->n_stencil == 5 || pr->n_stencil == 7 || pr->n_stencil == 9))
    return bad("n_stencil must be 1, 3, 5, 7 or 9");
  if (pr->n_stencil > 1 && !pr->neighbors) return bad("neighbors missing");
  if (!(pr->n_proj_per_atom == 0 || pr->n_proj_per_atom == 1 || pr->n_proj_per_atom == 4))
    return bad("n_proj_per_atom must be 0, 1 or 4");
  if (pr->n_atoms < 0 || (pr->n_atoms > 0 && (!pr->atom_dom || !pr->atom_pos || !pr->well_depth || !pr->well_width)))
    return bad("atom arrays missing");
  if (pr->n_atoms > 0 && pr->n_proj_per_atom > 0 && (!pr->proj_gamma || !pr->proj_width))
    return bad("projector arrays missing");
  if (!(pr->r_cut > 0)) return bad("r_cut must be positive");
  if (prm->cheb_degree < 2) return bad("cheb_degree must be >= 2");
  if (prm->max_iter < 0) return bad("max_iter must be >= 0");
  if (!(prm->tol >= 0)) return bad("tol must be >= 0");
  if (!(prm->precision == DGDFT_FP64 || prm->precision == DGDFT_MIXED)) return bad("unknown precision");
  const int M = pr->n_elem;
  P.M = M;
  P.n_stencil = pr->n_stencil;
  P.n_proj_per_atom = pr->n_proj_per_atom;
  P.r_cut = pr->r_cut;
  P.tot_grid = 0;
  for (int d = 0; d < pr->n_dom; d++) {
    for (int a = 0; a < 3; a++) {
      if (pr->dom_n[3 * d + a] < 1 || !(pr->dom_h[3 * d + a] > 0)) return bad("bad domain grid");
      if (pr->dom_n[3 * d + a] * pr->dom_h[3 * d + a] < 2 * pr->r_cut - 1e-12)
        return bad("every domain side must be >= 2 r_cut (unique minimum image)");
    }
    P.tot_grid = std::max<long long>(P.tot_grid, pr->dom_voff[d] + (long long)pr->dom_n[3 * d] * pr->dom_n[3 * d + 1] *
                                                                       pr->dom_n[3 * d + 2]);
  }
  for (int a = 0; a < pr->n_atoms; a++)
    if (pr->atom_dom[a] < 0 || pr->atom_dom[a] >= pr->n_dom) return bad("atom_dom out of range");
  P.desc.resize(M);
  int L = 0;
  for (int k = 0; k < M; k++) {
    ElemDesc& d = P.desc[k];
    d = ElemDesc{};
    d.dom = pr->elem_dom[k];
    if (d.dom < 0 || d.dom >= pr->n_dom) return bad("elem_dom out of range");
    for (int a = 0; a < 3; a++) {
      d.gn[a] = pr->dom_n[3 * d.dom + a];
      d.h[a] = pr->dom_h[3 * d.dom + a];
      d.qn[a] = pr->elem_Qn[3 * k + a];
      d.en[a] = pr->elem_En[3 * k + a];
      const int e0 = pr->elem_E0[3 * k + a];
      if (d.en[a] < 1 || d.en[a] > d.qn[a] || d.qn[a] > d.gn[a]) return bad("need 1 <= En <= Qn <= domain n");
      if ((d.qn[a] - d.en[a]) % 2) return bad("Qn - En must be even");
      if (e0 < 0 || e0 >= d.gn[a]) return bad("E0 out of range");
      d.eo[a] = (d.qn[a] - d.en[a]) / 2;
      d.q0[a] = ((e0 - d.eo[a]) % d.gn[a] + d.gn[a]) % d.gn[a];
    }
    if (d.qn[0] % 2 || d.qn[1] % 2) return unsup("Q extents in x and y must be even");
    if (d.qn[0] > 48 || d.qn[1] > 48 || d.qn[2] > kMaxLine) return unsup("Q extent too large (x,y <= 48, z <= 64)");
    if (!factor_line(d.qn[0], d.fx[0], d.fx[1]) || !factor_line(d.qn[1], d.fy[0], d.fy[1]) ||
        !factor_line(d.qn[2], d.fz[0], d.fz[1]))
      return unsup("Q extents must be products n1*n2 with n1, n2 in {1,2,3,4,5,6,8}");
    d.N = d.qn[0] * d.qn[1] * d.qn[2];
    d.NE = d.en[0] * d.en[1] * d.en[2];
    d.dV = d.h[0] * d.h[1] * d.h[2];
    d.n_eig = prm->n_eig[k];
    d.n_alb = prm->n_alb[k];
    d.n_blk = prm->n_blk ? prm->n_blk[k] : nblk_rule(d.n_eig);
    if (d.n_eig < 1 || d.n_alb < 1 || d.n_alb > d.n_eig || d.n_eig > d.n_blk) return bad("need 1 <= n_alb <= n_eig <= n_blk");
    if (d.n_blk > 96) return unsup("n_blk > 96");
    if (d.n_blk > d.N || d.n_eig > d.NE) return bad("block larger than the grid");
    d.gvoff = pr->dom_voff[d.dom];
    L = std::max(L, d.n_blk);
    if (pr->n_stencil > 1)
      for (int s = 0; s < pr->n_stencil; s++) {
        const int nb = pr->neighbors[k * pr->n_stencil + s];
        if (nb < -1 || nb >= M) return bad("neighbor id out of range");
      }
  }
  P.L = L;
  // atom boxes: Q regions, then E regions
  P.boxes.clear();
  P.dtab.clear();
  for (int k = 0; k < M; k++) {
    ElemDesc& d = P.desc[k];
    int ncol;
    atom_boxes(pr, d, d.q0, d.qn, d.pa_begin, d.pa_count, ncol, P);
    d.n_proj = ncol;
  }
  for (int k = 0; k < M; k++) {
    ElemDesc& d = P.desc[k];
    int e0[3];
    for (int a = 0; a < 3; a++) e0[a] = pr->elem_E0[3 * k + a];
    int ncol;
    atom_boxes(pr, d, e0, d.en, d.pe_begin, d.pe_count, ncol, P);
    d.n_proj_e = ncol;
  }
  if (P.dtab.empty()) P.dtab.push_back(0.0);
  P.n_qboxes = M > 0 ? P.desc[0].pe_begin : 0;
  P.fatoms.assign(P.boxes.size(), FusedAtomRec{});
  for (int k = 0; k < M; k++) {
    ElemDesc& d = P.desc[k];
    d.tab_off = d.pa_count ? P.boxes[d.pa_begin].toff : 0;
    d.tab_len = 0;
    for (int i = 0; i < d.pa_count; i++) {
      const AtomBox& b = P.boxes[d.pa_begin + i];
      FusedAtomRec& r = P.fatoms[d.pa_begin + i];
      for (int q = 0; q < 3; q++) { r.s[q] = b.s[q]; r.l[q] = b.l[q]; r.qn[q] = d.qn[q]; }
      r.dtab = b.toff;
      r.d0[0] = float(P.dtab[b.toff]);
      r.d0[1] = float(P.dtab[b.toff + b.l[0]]);
      r.d0[2] = float(P.dtab[b.toff + b.l[0] + b.l[1]]);
      r.inv2s2 = float(0.5 / (b.pwidth * b.pwidth));
      const int npa = pr->n_proj_per_atom;
      r.c[0] = npa >= 1 ? float(b.gamma[0] * b.ns * b.ns * d.dV) : 0.f;
      for (int q = 1; q < 4; q++) r.c[q] = npa == 4 ? float(b.gamma[q] * b.np * b.np * d.dV) : 0.f;
      d.tab_len = std::max(d.tab_len, b.toff - d.tab_off + b.l[0] + b.l[1] + b.l[2]);
    }
    for (int a = 0; a < 3; a++) {
      const double g = 2.0 * M_PI / (d.qn[a] * d.h[a]);
      d.kscale[a] = float(0.5 * g * g / double(d.N));
    }
  }
  // offsets
  for (int i = 0; i < kOffKinds; i++) { P.off[i].assign(M, 0); P.tot[i] = 0; }
  P.tot_p = P.tot_pe = 0;
  P.max_points = P.max_nblk = P.max_neig = P.max_nalb = 0;
  for (int k = 0; k < M; k++) {
    ElemDesc& d = P.desc[k];
    const long long hxn = (long long)d.qn[2] * d.qn[1] * (d.qn[0] / 2 + 1);
    const long long sz[kOffKinds] = {(long long)d.n_blk * d.N, (long long)d.n_eig * d.N, (long long)d.n_alb * d.NE,
                                     (long long)d.N, (long long)d.n_blk * hxn, (long long)d.n_eig * d.NE,
                                     (long long)d.NE};
    for (int i = 0; i < kOffKinds; i++) { P.off[i][k] = P.tot[i]; P.tot[i] += sz[i]; }
    d.xoff = P.off[OFF_X][k];
    d.eoff = P.off[OFF_E][k];
    d.aoff = P.off[OFF_A][k];
    d.voff = P.off[OFF_V][k];
    d.soff = P.off[OFF_S][k];
    d.poff = P.tot_p;
    P.tot_p += (long long)d.n_blk * d.n_proj;
    d.peoff = P.tot_pe;
    P.tot_pe += (long long)d.n_alb * d.n_proj_e;
    // DG faces: axes named by the stencil along which E does not span its domain
    const int nfa = P.n_stencil == 3 ? 1 : (P.n_stencil == 5 || P.n_stencil == 9 ? 2 : (P.n_stencil == 7 ? 3 : 0));
    d.face_mask = 0;
    d.fmax = 1;
    for (int a = 0; a < nfa; a++)
      if (d.en[a] < d.gn[a]) {
        d.face_mask |= 3 << (2 * a);
        d.fmax = std::max(d.fmax, d.NE / d.en[a]);
      }
    d.troff = P.tot_tr;
    if (d.face_mask) P.tot_tr += 6LL * 2 * d.n_alb * d.fmax;
    P.max_points = std::max(P.max_points, d.N);
    P.max_nblk = std::max(P.max_nblk, d.n_blk);
    P.max_neig = std::max(P.max_neig, d.n_eig);
    P.max_nalb = std::max(P.max_nalb, d.n_alb);
    P.max_pa = std::max(P.max_pa, d.pa_count);
    P.max_pe = std::max(P.max_pe, d.pe_count);
  }
  // face neighbours must share the transverse extents of the face (conforming partition)
  const int nfa = P.n_stencil == 3 ? 1 : (P.n_stencil == 5 || P.n_stencil == 9 ? 2 : (P.n_stencil == 7 ? 3 : 0));
  for (int k = 0; k < M; k++)
    for (int s = 1; s <= 2 * nfa; s++) {
      const int nb = pr->neighbors[k * pr->n_stencil + s];
      if (nb < 0) continue;
      const int axis = (s - 1) / 2;
      for (int a = 0; a < 3; a++)
        if (a != axis && P.desc[nb].en[a] != P.desc[k].en[a]) {
          msg = "face neighbours must have equal transverse E extents";
          return DGDFT_INVALID_ARG;
        }
    }
  // Q-shape groups
  std::map<std::tuple<int, int, int>, int> gid;
  P.hx.groups.clear();
  for (int k = 0; k < M; k++) {
    const ElemDesc& d = P.desc[k];
    auto key = std::make_tuple(d.qn[0], d.qn[1], d.qn[2]);
    auto it = gid.find(key);
    if (it == gid.end()) {
      ShapeGroup g{};
      g.qn[0] = d.qn[0]; g.qn[1] = d.qn[1]; g.qn[2] = d.qn[2];
      g.zchunk = 32;
      it = gid.emplace(key, int(P.hx.groups.size())).first;
      P.hx.groups.push_back(g);
    }
    ShapeGroup& g = P.hx.groups[it->second];
    if (g.elems.empty()) g.fused_ok = true;
    if (d.pa_count > kFusedAtomLimit) g.fused_ok = false;
    for (int ai = 0; ai < d.pa_count; ai++)
      for (int q = 0; q < 3; q++)
        if (P.boxes[d.pa_begin + ai].l[q] > 16) g.fused_ok = false;   // boxes must fit the 16^3 list slots
    g.elems.push_back(k);
    g.n_elems = int(g.elems.size());
    g.max_nblk = std::max(g.max_nblk, d.n_blk);
    g.max_neig = std::max(g.max_neig, d.n_eig);
    g.max_nalb = std::max(g.max_nalb, d.n_alb);
  }
  return DGDFT_OK;
}

}  // namespace dgdft
