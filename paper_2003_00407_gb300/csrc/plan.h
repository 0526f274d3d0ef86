// Per-call plan: element descriptors, atom support boxes, Q-shape groups and
// packed-buffer offsets, built on the host from the problem statement.
#pragma once
#include <string>
#include <vector>

#include "dgdft.h"
#include "kernels.h"

namespace dgdft {

enum OffKind { OFF_X = 0, OFF_E = 1, OFF_A = 2, OFF_V = 3, OFF_S = 4, OFF_FE = 5, OFF_VE = 6 };
constexpr int kOffKinds = 7;

struct Plan {
  int M = 0, L = 0, n_stencil = 1, n_proj_per_atom = 0;
  double r_cut = 0;
  std::vector<ElemDesc> desc;
  std::vector<AtomBox> boxes;   // Q boxes of all elements, then E boxes
  std::vector<double> dtab;
  std::vector<FusedAtomRec> fatoms;   // parallel to boxes (Q boxes filled)
  HxPlan hx;
  std::vector<long long> off[kOffKinds];
  long long tot[kOffKinds] = {0, 0, 0, 0, 0, 0, 0};
  long long tot_tr = 0;         // face traces
  long long tot_p = 0;          // projections [n_blk][n_proj] per element
  long long tot_pe = 0;         // E-projector overlaps [n_alb][n_proj_e] per element
  long long tot_grid = 0;       // points of all domains
  int max_points = 0, max_nblk = 0, max_neig = 0, max_nalb = 0, max_pa = 0, max_pe = 0;
  // device mirrors
  ElemDesc* d_desc = nullptr;
  AtomBox* d_boxes = nullptr;
  double* d_dtab = nullptr;
  ProjList plist{nullptr, nullptr};   // compact projector-point lists of the Q boxes (device)
  int n_qboxes = 0;                            // the Q boxes come first in `boxes`
  FusedAtomRec* d_fatoms = nullptr;
  long long* d_off[kOffKinds] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

// Validates the arguments and builds the plan.  Returns a dgdft_status.
int build_plan(const dgdft_problem* prob, const dgdft_alb_params* prm, Plan& P, std::string& msg);
bool factor_line(int n, int& n1, int& n2);

}  // namespace dgdft
