// Internal types shared by the kernels and the host orchestration of libdgdft.
// Layouts: every grid function is stored [z][y][x] with x fastest; a block of
// n vectors on Q_k is [n][N_k] (vector-major).  Packed buffers hold the blocks
// of all elements back to back at the offsets recorded in ElemDesc.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dgdft {

// Per-element geometry and buffer offsets (built on the host, mirrored on the device).
struct ElemDesc {
  int qn[3];        // Q extent (x, y, z)
  int en[3];        // E extent
  int eo[3];        // E offset inside Q
  int q0[3];        // global index of Q's first point, wrapped into [0, gn)
  int gn[3];        // domain grid
  int fx[2], fy[2], fz[2];   // line-FFT factorisations n = n1 * n2 per axis
  int N, NE;        // points of Q and of E
  int n_eig, n_blk, n_alb;
  int dom;
  int pa_begin, pa_count;    // atom-box records (wells and projectors) meeting Q
  int pe_begin, pe_count;    // atom-box records meeting E (DG projector overlaps)
  int n_proj;                // projector columns acting in Q (4 or 1 per atom record)
  int n_proj_e;              // projector columns meeting E
  double h[3];
  double dV;
  long long xoff;   // [n_blk][N] blocks in the work buffers (scalars)
  long long eoff;   // [n_eig][N] in the eigenvector output
  long long aoff;   // [n_alb][NE] in the ALB output
  long long voff;   // [N] in the V_Q buffers
  long long soff;   // [n_blk][qz][qy][qx/2+1] complex in the spectrum buffer
  long long gvoff;  // first point of the domain in v_extra / grad_v
  long long poff;   // [n_blk][n_proj] projections
  long long peoff;  // [n_alb][n_proj_e] projector overlaps on E (DG)
  long long troff;  // face traces [6 faces][2 kinds][n_alb][fmax] (DG)
  int fmax;         // largest face (points) of E
  int face_mask;    // bit (axis*2 + side) set when that face carries DG terms
  int tab_off, tab_len;  // the element's Q-box displacement tables in dtab (contiguous)
  float kscale[3];  // 1/2 (2 pi / (n_a h_a))^2 / N: kinetic multiplier per m_a^2
};

// Record of an atom box meeting Q for the fused FP32 Chebyshev kernel (parallel to the Q boxes).
// The kernel reads the box's projector points from a compact list (see ProjList); the record holds what
// turns the list's moments into the four projector overlaps and back.
struct FusedAtomRec {
  int s[3], l[3];   // box start (cyclic, Q-local) and extent per axis
  int dtab;         // first entry of the box's displacement tables in the plan's dtab (x, then y, then z)
  int qn[3];        // Q extent of the element (smem row layout of the fused kernel)
  float inv2s2;     // 1 / (2 sigma^2) of the projector radial Gaussian
  float c[4];       // gamma_l N_l^2 dV for s, px, py, pz (0 when absent)
  float d0[3];      // displacement (bohr) of the box's first point along x, y, z; point i: d0 + i h
};

// Compact projector-point lists, one slot of kProjCap entries per fused atom record: the box points of
// Q inside the support ball in (z, y, x) order, one 64-bit entry (bits of g, w) per point:
// g = exp(-d^2 / 2 sigma^2) (1 - d^2/r_cut^2)^3 and
// w = (float index of the point in the fused kernel's row layout) | ix << 16 | iy << 20 | iz << 24;
// n[2r] = number of points of record r, n[2r + 1] = 0.  For Q shapes whose vectors are split over a CTA
// pair by plane parity: the points on even z planes first, then those on odd planes, indexed in the row
// layout of the planes of their parity (plane z at slot z / 2), n[2r] and n[2r + 1] their numbers.
constexpr int kProjCap = 4096;
struct ProjList {
  uint2* gw;
  int* n;
};

// An atom whose support box meets a region (Q or E) of one element.  The box
// is, per axis, a cyclic run of l[a] region-local indices starting at s[a];
// dtab[toff + ...] holds the minimum-image displacement (bohr) of each index
// along x, then y, then z.
struct AtomBox {
  int atom;         // global atom id
  int s[3], l[3];
  int toff;
  int col;          // first projector column of this atom in the element's projection array
  double depth, wwidth;      // local well
  double pwidth, ns, np;     // projector radial sigma and norms
  double gamma[4];
};

enum Status {
  ST_OK = 0, ST_INVALID_ARG = 1, ST_OUT_OF_MEMORY = 2, ST_NOT_CONVERGED = 3,
  ST_CHOLESKY_FAIL = 4, ST_BAD_INPUT = 5, ST_TIMEOUT = 6, ST_CUDA_ERROR = 7, ST_UNSUPPORTED = 8
};

// Device-side per-element flags (bit field in an int array)
enum ElemFlag { EF_ACTIVE = 1, EF_CHOL_SHIFT = 2, EF_CHOL_FAIL = 4, EF_BAD = 8, EF_JACOBI_CAP = 16 };

template <typename T> struct cplx { T re, im; };

}  // namespace dgdft
