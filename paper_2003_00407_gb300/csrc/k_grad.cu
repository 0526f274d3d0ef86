// Band energy and its Hellmann-Feynman gradient (local analogue of Eq. hfforce).
//   E_k = sum_j 2 f_j lambda_j,  f_j = 1/(1 + exp((lambda_j - mu_k)/kT)),  sum_j 2 f_j = N_el,k
//   dE/dtheta = sum_j w_j <phi_j, dH/dtheta phi_j>,  w_j = 2 [f_j + f'_j (lambda_j - mu_bar)],
//   mu_bar = sum lambda f' / sum f'.
// dE/dV(g) sums w_j phi_j^2 dV over the Q points mapped to g; dE/dR_I adds the
// well term sum_q rho(q) dV_I/dR_I and the projector term
// 2 sum_l gamma_l <phi_j, b_l> <phi_j, db_l/dR_I> weighted by w_j.
#include "kernels.h"

namespace dgdft {

constexpr int kGChunk = 768;   // box points cached per pass
constexpr int kMaxEig = 96;

__device__ __forceinline__ double fermi_fn(double lam, double mu, double kT) {
  double x = (lam - mu) / kT;
  x = fmin(fmax(x, -700.0), 700.0);
  return 1.0 / (1.0 + exp(x));
}

__global__ void k_fermi_weights(BatchArgs b, const double* theta, int ld, const double* n_el, double kT, double* w,
                                double* energy, int* flags) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.M) return;
  const int n = b.desc[k].n_eig;
  const double* lam = theta + (long long)k * ld;
  double lmin = lam[0], lmax = lam[0];
  for (int j = 1; j < n; j++) { lmin = fmin(lmin, lam[j]); lmax = fmax(lmax, lam[j]); }
  double lo = lmin - 50.0 * kT - 1.0, hi = lmax + 50.0 * kT + 1.0;
  for (int it = 0; it < 200; it++) {
    const double mid = 0.5 * (lo + hi);
    double s = 0.0;
    for (int j = 0; j < n; j++) s += 2.0 * fermi_fn(lam[j], mid, kT);
    if (s > n_el[k]) hi = mid; else lo = mid;
  }
  const double mu = 0.5 * (lo + hi);
  double E = 0.0, sfp = 0.0, slfp = 0.0;
  for (int j = 0; j < n; j++) {
    const double f = fermi_fn(lam[j], mu, kT), fp = -f * (1.0 - f) / kT;
    E += 2.0 * f * lam[j];
    sfp += fp;
    slfp += lam[j] * fp;
  }
  const double mubar = sfp != 0.0 ? slfp / sfp : 0.0;
  for (int j = 0; j < n; j++) {
    const double f = fermi_fn(lam[j], mu, kT), fp = -f * (1.0 - f) / kT;
    w[(long long)k * ld + j] = 2.0 * (f + fp * (lam[j] - mubar));
  }
  if (fermi_fn(lam[n - 1], mu, kT) >= 1e-12) atomicOr(&flags[k], EF_BAD);
  energy[k] = E;
}

void launch_fermi_weights(const BatchArgs& b, const double* theta, int ld, const double* n_el, double kT, double* w,
                          double* energy, int* flags, cudaStream_t st) {
  count_launch(); k_fermi_weights<<<(b.M + 127) / 128, 128, 0, st>>>(b, theta, ld, n_el, kT, w, energy, flags);
}

// rho(q) = sum_j w_j phi_j(q)^2 dV on Q, scattered onto the domain grid
__global__ void k_density_scatter(BatchArgs b, const double* Phi, const long long* po, const double* w, int ld,
                                  double* rho, const long long* ro, double* grad_v) {
  const int k = blockIdx.y;
  const ElemDesc& d = b.desc[k];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.N) return;
  const double* pk = Phi + po[k];
  double s = 0.0;
  for (int j = 0; j < d.n_eig; j++) {
    const double v = pk[(long long)j * d.N + q];
    s += w[(long long)k * ld + j] * v * v;
  }
  s *= d.dV;
  rho[ro[k] + q] = s;
  const int x = q % d.qn[0], y = (q / d.qn[0]) % d.qn[1], z = q / (d.qn[0] * d.qn[1]);
  const int gx = (d.q0[0] + x) % d.gn[0], gy = (d.q0[1] + y) % d.gn[1], gz = (d.q0[2] + z) % d.gn[2];
  atomicAdd(&grad_v[d.gvoff + ((long long)gz * d.gn[1] + gy) * d.gn[0] + gx], s);
}

void launch_density_scatter(const BatchArgs& b, const double* Phi, const long long* po, const double* w, int ld,
                            double* rho, const long long* ro, double* grad_v, cudaStream_t st) {
  count_launch(); k_density_scatter<<<dim3((g_max_points + 255) / 256, b.M), 256, 0, st>>>(b, Phi, po, w, ld, rho, ro, grad_v);
}

// g = exp(-d^2/2 s^2) (1 - d^2/rc^2)^3 and dg/dd_alpha = g_gauss d_alpha (-(1-s2)^3/s^2 - 6 (1-s2)^2/rc^2)
__device__ __forceinline__ void gauss_taper(double dx, double dy, double dz, double sig, double inv_rc2, double& g,
                                            double& gx, double& gy, double& gz) {
  const double d2 = dx * dx + dy * dy + dz * dz;
  const double one = 1.0 - d2 * inv_rc2;
  if (one <= 0.0) { g = gx = gy = gz = 0.0; return; }
  const double ga = exp(-d2 / (2.0 * sig * sig));
  g = ga * one * one * one;
  const double common = ga * (-(one * one * one) / (sig * sig) - 6.0 * one * one * inv_rc2);
  gx = common * dx; gy = common * dy; gz = common * dz;
}

__global__ void __launch_bounds__(256) k_atom_forces(BatchArgs b, const AtomBox* boxes, const double* dtab,
                                                     const double* Phi, const long long* po, const double* w, int ld,
                                                     const double* rho, const long long* ro, double r_cut, int npa,
                                                     double* grad_R) {
  const int k = blockIdx.y;
  const ElemDesc& d = b.desc[k];
  const int bi = blockIdx.x;
  if (bi >= d.pa_count) return;
  const AtomBox& bx = boxes[d.pa_begin + bi];
  __shared__ double cg[kGChunk][4];   // projector radial g and dg/dd
  __shared__ int qidx[kGChunk];
  __shared__ double facc[3];
  __shared__ double ov[kMaxEig][16];  // per eigenvector: <phi,b_l> (4) and <phi, db_l/dR_a> (12) over the whole box
  if (threadIdx.x < 3) facc[threadIdx.x] = 0.0;
  for (int i = threadIdx.x; i < kMaxEig * 16; i += blockDim.x) (&ov[0][0])[i] = 0.0;
  const double* t = dtab + bx.toff;
  const int npts = bx.l[0] * bx.l[1] * bx.l[2];
  const double inv_rc2 = 1.0 / (r_cut * r_cut);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const double* pk = Phi + po[k];
  double fw[3] = {0.0, 0.0, 0.0};   // per-thread well term
  double fp[3] = {0.0, 0.0, 0.0};   // per-thread projector term
  for (int c0 = 0; c0 < npts; c0 += kGChunk) {
    const int cn = min(kGChunk, npts - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < cn; i += blockDim.x) {
      const int p = c0 + i;
      const int ix = p % bx.l[0], iy = (p / bx.l[0]) % bx.l[1], iz = p / (bx.l[0] * bx.l[1]);
      int x = bx.s[0] + ix; if (x >= d.qn[0]) x -= d.qn[0];
      int y = bx.s[1] + iy; if (y >= d.qn[1]) y -= d.qn[1];
      int z = bx.s[2] + iz; if (z >= d.qn[2]) z -= d.qn[2];
      const int q = (z * d.qn[1] + y) * d.qn[0] + x;
      const double dx = t[ix], dy = t[bx.l[0] + iy], dz = t[bx.l[0] + bx.l[1] + iz];
      double g, gx, gy, gz;
      gauss_taper(dx, dy, dz, bx.wwidth, inv_rc2, g, gx, gy, gz);
      const double r = rho[ro[k] + q];
      fw[0] += bx.depth * r * gx;   // V_I = -D g  =>  dV_I/dR = +D dg/dd
      fw[1] += bx.depth * r * gy;
      fw[2] += bx.depth * r * gz;
      gauss_taper(dx, dy, dz, bx.pwidth, inv_rc2, g, gx, gy, gz);
      cg[i][0] = g; cg[i][1] = gx; cg[i][2] = gy; cg[i][3] = gz;
      qidx[i] = q;
    }
    __syncthreads();
    if (npa == 0) continue;
    // projector term per eigenvector: 4 overlaps <phi,b_l> and 12 <phi, db_l/dR_a>
    for (int j = warp; j < d.n_eig; j += nw) {
      const double* pj = pk + (long long)j * d.N;
      double pb[4] = {0, 0, 0, 0}, pd[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      for (int i = lane; i < cn; i += 32) {
        const double g = cg[i][0];
        if (g == 0.0 && cg[i][1] == 0.0) continue;
        const int p = c0 + i;
        const int ix = p % bx.l[0], iy = (p / bx.l[0]) % bx.l[1], iz = p / (bx.l[0] * bx.l[1]);
        const double dd[3] = {t[ix], t[bx.l[0] + iy], t[bx.l[0] + bx.l[1] + iz]};
        const double v = pj[qidx[i]];
        const double dg[3] = {cg[i][1], cg[i][2], cg[i][3]};
        pb[0] += v * g;
        for (int a = 0; a < 3; a++) pd[0][a] -= v * dg[a];     // db_s/dR = -N_s dg/dd
        if (npa == 4)
          for (int be = 0; be < 3; be++) {
            pb[1 + be] += v * dd[be] * g;
            for (int a = 0; a < 3; a++) pd[1 + be][a] -= v * ((a == be ? g : 0.0) + dd[be] * dg[a]);
          }
      }
      for (int o = 16; o > 0; o >>= 1) {
        for (int l = 0; l < 4; l++) {
          pb[l] += __shfl_xor_sync(0xffffffffu, pb[l], o);
          for (int a = 0; a < 3; a++) pd[l][a] += __shfl_xor_sync(0xffffffffu, pd[l][a], o);
        }
      }
      if (lane == 0) {  // the same warp owns eigenvector j in every chunk
        for (int l = 0; l < 4; l++) {
          ov[j][l] += pb[l];
          for (int a = 0; a < 3; a++) ov[j][4 + 3 * l + a] += pd[l][a];
        }
      }
    }
  }
  __syncthreads();
  if (npa > 0)
    for (int j = threadIdx.x; j < d.n_eig; j += blockDim.x) {
      const double wj = w[(long long)k * ld + j];
      for (int l = 0; l < npa; l++) {
        const double nrm = (l == 0 ? bx.ns : bx.np) * d.dV;
        for (int a = 0; a < 3; a++) fp[a] += wj * 2.0 * bx.gamma[l] * (ov[j][l] * nrm) * (ov[j][4 + 3 * l + a] * nrm);
      }
    }
  for (int a = 0; a < 3; a++) {
    double v = fw[a] + fp[a];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) atomicAdd(&facc[a], v);
  }
  __syncthreads();
  if (threadIdx.x < 3) atomicAdd(&grad_R[(long long)bx.atom * 3 + threadIdx.x], facc[threadIdx.x]);
}

void launch_atom_forces(const BatchArgs& b, const AtomBox* boxes, const double* dtab, const double* Phi,
                        const long long* po, const double* w, int ld, const double* rho, const long long* ro,
                        double r_cut, int n_proj_per_atom, double* grad_R, int max_boxes, cudaStream_t st) {
  if (max_boxes <= 0) return;
  count_launch(); k_atom_forces<<<dim3(max_boxes, b.M), 256, 0, st>>>(b, boxes, dtab, Phi, po, w, ld, rho, ro, r_cut,
                                                      n_proj_per_atom, grad_R);
}

}  // namespace dgdft
