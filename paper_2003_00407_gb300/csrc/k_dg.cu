// DG Hamiltonian ingredients and blocks (Eq. DGHamiltonian).
//
// Readings (standard symmetric interior-penalty DG on the cell-centred
// element partition): faces lie half a spacing outside E's end points; an
// ALB is the restriction of the trigonometric interpolant psi = Phi^Q C on
// Q, so face values and normal derivatives apply 1D weights along the normal
// line of Q (Nyquist term dropped); with n from L (the -axis element) to R,
// [[u]] = u_L - u_R and {{d u}} = (d u_L + d u_R)/2 give per face
//   v,u in L: -1/4 v du - 1/4 dv u + alpha v u     v,u in R: +1/4 v du + 1/4 dv u + alpha v u
//   v in L, u in R: -1/4 v du + 1/4 dv u - alpha v u   (v in R, u in L: the transpose).
#include "kernels.h"

namespace dgdft {

constexpr int kMaxAlb = 96;
constexpr int kChunk = 2048;  // box points cached per pass

// ---- projector overlaps on E: PE[j][col+l] = dV sum_{e in E} b_l(e) A_j(e) ----
__global__ void __launch_bounds__(256) k_proj_overlap(BatchArgs b, const AtomBox* boxes, const double* dtab,
                                                      const double* A, const long long* ao, double r_cut, int npa,
                                                      double* PE) {
  const int k = blockIdx.y;
  const ElemDesc& d = b.desc[k];
  const int bi = blockIdx.x;
  if (bi >= d.pe_count || npa == 0) return;
  const AtomBox& bx = boxes[d.pe_begin + bi];
  __shared__ double g[kChunk];
  __shared__ int eidx[kChunk];
  __shared__ double acc[kMaxAlb][4];
  for (int i = threadIdx.x; i < kMaxAlb * 4; i += blockDim.x) (&acc[0][0])[i] = 0.0;
  const double* t = dtab + bx.toff;
  const int npts = bx.l[0] * bx.l[1] * bx.l[2];
  const double inv_rc2 = 1.0 / (r_cut * r_cut), inv2s2 = 0.5 / (bx.pwidth * bx.pwidth);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const double* Ak = A + ao[k];
  for (int c0 = 0; c0 < npts; c0 += kChunk) {
    const int cn = min(kChunk, npts - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < cn; i += blockDim.x) {
      const int p = c0 + i;
      const int ix = p % bx.l[0], iy = (p / bx.l[0]) % bx.l[1], iz = p / (bx.l[0] * bx.l[1]);
      int ex = bx.s[0] + ix; if (ex >= d.en[0]) ex -= d.en[0];
      int ey = bx.s[1] + iy; if (ey >= d.en[1]) ey -= d.en[1];
      int ez = bx.s[2] + iz; if (ez >= d.en[2]) ez -= d.en[2];
      const double dx = t[ix], dy = t[bx.l[0] + iy], dz = t[bx.l[0] + bx.l[1] + iz];
      const double d2 = dx * dx + dy * dy + dz * dz;
      const double u = 1.0 - d2 * inv_rc2;
      g[i] = u > 0.0 ? exp(-d2 * inv2s2) * u * u * u : 0.0;
      eidx[i] = (ez * d.en[1] + ey) * d.en[0] + ex;
    }
    __syncthreads();
    for (int j = warp; j < d.n_alb; j += nw) {
      const double* Aj = Ak + (long long)j * d.NE;
      double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      for (int i = lane; i < cn; i += 32) {
        const double gv = g[i];
        if (gv == 0.0) continue;
        const int p = c0 + i;
        const int ix = p % bx.l[0], iy = (p / bx.l[0]) % bx.l[1], iz = p / (bx.l[0] * bx.l[1]);
        const double v = Aj[eidx[i]] * gv;
        s0 += v;
        s1 += v * t[ix];
        s2 += v * t[bx.l[0] + iy];
        s3 += v * t[bx.l[0] + bx.l[1] + iz];
      }
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
      }
      if (lane == 0) { acc[j][0] += s0; acc[j][1] += s1; acc[j][2] += s2; acc[j][3] += s3; }
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < d.n_alb * npa; idx += blockDim.x) {
    const int j = idx / npa, l = idx % npa;
    PE[d.peoff + (long long)j * d.n_proj_e + bx.col + l] = acc[j][l] * (l == 0 ? bx.ns : bx.np) * d.dV;
  }
}

void launch_proj_overlap(const BatchArgs& b, const AtomBox* boxes, const double* dtab, const double* A,
                         const long long* ao, double r_cut, int n_proj_per_atom, double* PE, int max_boxes,
                         cudaStream_t st) {
  if (max_boxes <= 0 || n_proj_per_atom == 0) return;
  count_launch(); k_proj_overlap<<<dim3(max_boxes, b.M), 256, 0, st>>>(b, boxes, dtab, A, ao, r_cut, n_proj_per_atom, PE);
}

// ---- face traces of psi = Phi^Q C on Q (Psi [n_alb][N] per element) ----
// TR[troff + ((face*2 + kind) * n_alb + j) * fmax + f], face = 2*axis + (side > 0), kind 0 value, 1 derivative
__global__ void __launch_bounds__(256) k_face_traces(BatchArgs b, const double* Psi, const long long* po, double* TR) {
  const int k = blockIdx.z, face = blockIdx.y, j = blockIdx.x;
  const ElemDesc& d = b.desc[k];
  if (j >= d.n_alb || !((d.face_mask >> face) & 1)) return;
  const int axis = face >> 1, side = face & 1;
  const int n = d.qn[axis];
  __shared__ double wv[kMaxLine], wd[kMaxLine];
  const double h = d.h[axis];
  const double xf = side ? d.eo[axis] + d.en[axis] - 0.5 : d.eo[axis] - 0.5;
  const int mmax = (n % 2) ? (n - 1) / 2 : n / 2 - 1;
  const double twopi = 6.283185307179586476925;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double delta = (xf - i) * h;
    double sv = 1.0, sd = 0.0;
    for (int m = 1; m <= mmax; m++) {
      const double G = twopi * m / (n * h);
      double sn, cs;
      sincos(G * delta, &sn, &cs);
      sv += 2.0 * cs;
      sd -= 2.0 * G * sn;
    }
    wv[i] = sv / n;
    wd[i] = sd / n;
  }
  __syncthreads();
  // transverse axes (in [z][y][x] order of the remaining two): t1 slow, t0 fast
  const int a0 = axis == 0 ? 1 : 0;
  const int a1 = axis == 2 ? 1 : 2;
  const int F = d.en[a0] * d.en[a1];
  const int st[3] = {1, d.qn[0], d.qn[0] * d.qn[1]};
  const double* pj = Psi + po[k] + (long long)j * d.N;
  double* tv = TR + d.troff + ((long long)(face * 2 + 0) * d.n_alb + j) * d.fmax;
  double* td = TR + d.troff + ((long long)(face * 2 + 1) * d.n_alb + j) * d.fmax;
  for (int f = threadIdx.x; f < F; f += blockDim.x) {
    const int i0 = f % d.en[a0], i1 = f / d.en[a0];
    const long long base = (long long)(i0 + d.eo[a0]) * st[a0] + (long long)(i1 + d.eo[a1]) * st[a1];
    double sv = 0.0, sd = 0.0;
    for (int i = 0; i < n; i++) {
      const double v = pj[base + (long long)i * st[axis]];
      sv += wv[i] * v;
      sd += wd[i] * v;
    }
    tv[f] = sv;
    td[f] = sd;
  }
}

void launch_face_traces(const BatchArgs& b, const double* Psi, const long long* po, double* TR, cudaStream_t st) {
  count_launch(); k_face_traces<<<dim3(g_max_nalb, 6, b.M), 256, 0, st>>>(b, Psi, po, TR);
}

// ---- blocks: slot s of element k, rows = test ALBs of k, columns = trial ALBs of neighbour n ----
constexpr int kFT = 12;  // face points per tile (static shared memory < 48 KB)
__global__ void __launch_bounds__(256) k_dg_blocks(BatchArgs b, const int* neighbors, int n_stencil,
                                                   const double* TR, const double* PE, const AtomBox* boxes, int npa,
                                                   const double* KV, int ld, double alpha, double* blocks) {
  const int k = blockIdx.y, s = blockIdx.x;
  const ElemDesc& dk = b.desc[k];
  const int n = s == 0 ? k : neighbors[k * n_stencil + s];
  double* out = blocks + ((long long)k * n_stencil + s) * ld * ld;
  if (n < 0) {
    for (int i = threadIdx.x; i < ld * ld; i += blockDim.x) out[i] = 0.0;
    return;
  }
  const ElemDesc& dn = b.desc[n];
  const int nk = dk.n_alb, nn = dn.n_alb;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[6][6];
#pragma unroll
  for (int r = 0; r < 6; r++)
#pragma unroll
    for (int c = 0; c < 6; c++) acc[r][c] = 0.0;
  __shared__ double sVk[kFT][kMaxAlb + 1], sDk[kFT][kMaxAlb + 1], sVn[kFT][kMaxAlb + 1], sDn[kFT][kMaxAlb + 1];
  const int nfa_slots = n_stencil == 3 ? 2 : (n_stencil == 5 || n_stencil == 9 ? 4 : (n_stencil == 7 ? 6 : 0));
  // faces contributing to this slot: (face of k, face of n, c_vd, c_dv, c_vv)
  for (int fi = 0; fi < 6; fi++) {
    int fk = -1, fn = -1;
    double c1 = 0, c2 = 0, c3 = 0;
    if (s == 0) {
      if (!((dk.face_mask >> fi) & 1)) continue;
      fk = fn = fi;
      const bool low = (fi & 1) == 0;  // k is R on its low face
      c1 = c2 = low ? 0.25 : -0.25;
      c3 = alpha;
    } else {
      if (fi > 0 || s > nfa_slots) continue;
      const int axis = (s - 1) >> 1, high = (s - 1) & 1;
      fk = 2 * axis + high;
      fn = 2 * axis + (1 - high);
      if (!((dk.face_mask >> fk) & 1) || !((dn.face_mask >> fn) & 1)) continue;
      if (high) { c1 = -0.25; c2 = 0.25; }   // k = L, n = R
      else { c1 = 0.25; c2 = -0.25; }        // k = R, n = L
      c3 = -alpha;
    }
    const int axis = fk >> 1;
    const double dA = axis == 0 ? dk.h[1] * dk.h[2] : (axis == 1 ? dk.h[0] * dk.h[2] : dk.h[0] * dk.h[1]);
    const int F = dk.NE / dk.en[axis];
    const double* Vk = TR + dk.troff + (long long)(fk * 2 + 0) * nk * dk.fmax;
    const double* Dk = TR + dk.troff + (long long)(fk * 2 + 1) * nk * dk.fmax;
    const double* Vn = TR + dn.troff + (long long)(fn * 2 + 0) * nn * dn.fmax;
    const double* Dn = TR + dn.troff + (long long)(fn * 2 + 1) * nn * dn.fmax;
    for (int f0 = 0; f0 < F; f0 += kFT) {
      __syncthreads();
      for (int idx = threadIdx.x; idx < kFT * kMaxAlb; idx += blockDim.x) {
        const int ff = idx % kFT, j = idx / kFT;
        const int f = f0 + ff;
        const bool okf = f < F;
        sVk[ff][j] = (okf && j < nk) ? Vk[(long long)j * dk.fmax + f] : 0.0;
        sDk[ff][j] = (okf && j < nk) ? Dk[(long long)j * dk.fmax + f] : 0.0;
        sVn[ff][j] = (okf && j < nn) ? Vn[(long long)j * dn.fmax + f] : 0.0;
        sDn[ff][j] = (okf && j < nn) ? Dn[(long long)j * dn.fmax + f] : 0.0;
      }
      __syncthreads();
#pragma unroll 4
      for (int ff = 0; ff < kFT; ff++) {
        double av[6], ad[6], bv[6], bd[6];
#pragma unroll
        for (int r = 0; r < 6; r++) { av[r] = sVk[ff][ty + 16 * r]; ad[r] = sDk[ff][ty + 16 * r]; }
#pragma unroll
        for (int c = 0; c < 6; c++) { bv[c] = sVn[ff][tx + 16 * c]; bd[c] = sDn[ff][tx + 16 * c]; }
#pragma unroll
        for (int r = 0; r < 6; r++)
#pragma unroll
          for (int c = 0; c < 6; c++) acc[r][c] += dA * (c1 * av[r] * bd[c] + c2 * ad[r] * bv[c] + c3 * av[r] * bv[c]);
      }
    }
  }
  // nonlocal coupling, in the first slot naming the pair
  bool first = true;
  for (int s2 = 0; s2 < s; s2++)
    if ((s2 == 0 ? k : neighbors[k * n_stencil + s2]) == n) first = false;
  __shared__ int pk[128], pn[128];
  __shared__ double pg[128][4];
  __shared__ int npair;
  if (threadIdx.x == 0) {
    int m = 0;
    if (first && npa > 0)
      for (int a = 0; a < dk.pe_count && m < 128; a++) {
        const AtomBox& ba = boxes[dk.pe_begin + a];
        for (int c = 0; c < dn.pe_count; c++) {
          const AtomBox& bc = boxes[dn.pe_begin + c];
          if (bc.atom == ba.atom) {
            pk[m] = ba.col; pn[m] = bc.col;
            for (int l = 0; l < 4; l++) pg[m][l] = ba.gamma[l];
            m++;
            break;
          }
        }
      }
    npair = m;
  }
  __syncthreads();
  const double* Pk = PE + dk.peoff;
  const double* Pn = PE + dn.peoff;
  for (int r = 0; r < 6; r++) {
    const int i = ty + 16 * r;
    for (int c = 0; c < 6; c++) {
      const int j = tx + 16 * c;
      if (i >= nk || j >= nn) continue;
      double v = acc[r][c];
      for (int m = 0; m < npair; m++)
        for (int l = 0; l < npa; l++)
          v += pg[m][l] * Pk[(long long)i * dk.n_proj_e + pk[m] + l] * Pn[(long long)j * dn.n_proj_e + pn[m] + l];
      if (s == 0) v += KV[(long long)k * ld * ld + i * ld + j];
      acc[r][c] = v;
    }
  }
  for (int idx = threadIdx.x; idx < ld * ld; idx += blockDim.x) {
    const int i = idx / ld, j = idx % ld;
    if (i >= nk || j >= nn) out[idx] = 0.0;
  }
#pragma unroll
  for (int r = 0; r < 6; r++)
#pragma unroll
    for (int c = 0; c < 6; c++) {
      const int i = ty + 16 * r, j = tx + 16 * c;
      if (i < nk && j < nn) out[i * ld + j] = acc[r][c];
    }
}

void launch_dg_blocks(const BatchArgs& b, const int* neighbors, int n_stencil, const double* TR, const double* PE,
                      const AtomBox* boxes, int n_proj_per_atom, const double* KV, int ld, double alpha,
                      double* blocks, cudaStream_t st) {
  count_launch(); k_dg_blocks<<<dim3(n_stencil, b.M), 256, 0, st>>>(b, neighbors, n_stencil, TR, PE, boxes, n_proj_per_atom, KV, ld,
                                                    alpha, blocks);
}

}  // namespace dgdft
