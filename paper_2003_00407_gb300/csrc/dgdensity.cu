// Electron density, band energy and Hellmann-Feynman forces of the DG solution (Sec. II.A: Eq. density
// with the diagonal blocks of the density matrix, Eq. densitymatrix; the total-energy form Eq. DGvar on
// the DG eigenpairs; Eq. hfforce for this model: local wells and Kleinman-Bylander projectors, with the
// ALBs held fixed).  FP64.
//
//   f_i Fermi-Dirac at kT with mu fixed by sum_i 2 f_i = N_e;  E = sum_i 2 f_i eps_i
//   psi_i = sum_{k,a} c_{i,ka} phi_{k,a}  (phi_{k,a} supported on E_k)
//   rho(r) = sum_i 2 f_i psi_i(r)^2 = sum_{a,b} phi_{k,a}(r) P_{ka,kb} phi_{k,b}(r) on E_k
//   dE/dR_I = sum_i w_i [ <psi_i, dV_I/dR_I psi_i> + 2 sum_l gamma_l <psi_i, b_l> <psi_i, db_l/dR_I> ],
//   w_i = 2 [f_i + f'_i (eps_i - mu_bar)],  mu_bar = sum eps f' / sum f'   (force = -dE/dR).
#include <algorithm>
#include <string>
#include <vector>

#include "context.h"
#include "dgdft.h"
#include "kernels.h"
#include "plan.h"

namespace dgdft {

int fail(dgdft_ctx* c, int code, const std::string& msg);
void* ws(dgdft_ctx* ctx, const std::string& name, size_t bytes);

namespace {

constexpr int kMaxStates = 96;
constexpr int kDChunk = 512;   // box points cached per pass

__device__ __forceinline__ double fermi_dg(double lam, double mu, double kT) {
  double x = (lam - mu) / kT;
  x = fmin(fmax(x, -700.0), 700.0);
  return 1.0 / (1.0 + exp(x));
}

// mu by bisection, occupations occ_i = 2 f_i, Hellmann-Feynman weights w_i, E and mu -> em[0..1]
__global__ void k_dg_fermi(const double* eps, int n, double n_el, double kT, double* occ, double* w, double* em,
                           int* bad) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double lmin = eps[0], lmax = eps[0];
  for (int j = 1; j < n; j++) { lmin = fmin(lmin, eps[j]); lmax = fmax(lmax, eps[j]); }
  double lo = lmin - 50.0 * kT - 1.0, hi = lmax + 50.0 * kT + 1.0;
  for (int it = 0; it < 200; it++) {
    const double mid = 0.5 * (lo + hi);
    double s = 0.0;
    for (int j = 0; j < n; j++) s += 2.0 * fermi_dg(eps[j], mid, kT);
    if (s > n_el) hi = mid; else lo = mid;
  }
  const double mu = 0.5 * (lo + hi);
  double E = 0.0, sfp = 0.0, slfp = 0.0;
  for (int j = 0; j < n; j++) {
    const double f = fermi_dg(eps[j], mu, kT), fp = -f * (1.0 - f) / kT;
    E += 2.0 * f * eps[j];
    sfp += fp;
    slfp += eps[j] * fp;
  }
  const double mubar = sfp != 0.0 ? slfp / sfp : 0.0;
  for (int j = 0; j < n; j++) {
    const double f = fermi_dg(eps[j], mu, kT), fp = -f * (1.0 - f) / kT;
    occ[j] = 2.0 * f;
    w[j] = 2.0 * (f + fp * (eps[j] - mubar));
  }
  em[0] = E;
  em[1] = mu;
  *bad = (!(E == E) || fermi_dg(eps[n - 1], mu, kT) >= 1e-12) ? 1 : 0;
}

// psi_i on E_k: Psi[pso_k + i*NE + e] = sum_a C[i][off_k + a] A_k[a][e]; grid (64-point tiles, M),
// 256 threads: point p = tid % 64 of the tile, states i = tid / 64 (mod 4); C_k and the A tile in shared memory
constexpr int kPsiTile = 64;
__global__ void __launch_bounds__(256) k_dg_psi(const ElemDesc* desc, const double* A, const long long* ao,
                                                const double* C, int Nb, int n, const int* off, double* Psi,
                                                const long long* pso) {
  const int k = blockIdx.y;
  const ElemDesc& d = desc[k];
  const int e0 = blockIdx.x * kPsiTile;
  if (e0 >= d.NE) return;
  extern __shared__ double sm[];
  const int na = d.n_alb;
  double* sC = sm;                       // [n][na]
  double* sA = sm + n * na;              // [na][kPsiTile]
  for (int idx = threadIdx.x; idx < n * na; idx += blockDim.x)
    sC[idx] = C[(long long)(idx / na) * Nb + off[k] + idx % na];
  const double* Ak = A + ao[k];
  for (int idx = threadIdx.x; idx < na * kPsiTile; idx += blockDim.x) {
    const int a = idx / kPsiTile, p = idx % kPsiTile;
    sA[idx] = e0 + p < d.NE ? Ak[(long long)a * d.NE + e0 + p] : 0.0;
  }
  __syncthreads();
  const int p = threadIdx.x % kPsiTile, g = threadIdx.x / kPsiTile;
  if (e0 + p >= d.NE) return;
  double* out = Psi + pso[k];
  for (int i = g; i < n; i += blockDim.x / kPsiTile) {
    double s = 0.0;
    for (int a = 0; a < na; a++) s = fma(sC[i * na + a], sA[a * kPsiTile + p], s);
    out[(long long)i * d.NE + e0 + p] = s;
  }
}

// rho = sum_i occ_i psi_i^2 onto the domain grid (E_k points), rho_w = sum_i w_i psi_i^2 on E_k
__global__ void k_dg_rho(const ElemDesc* desc, const double* Psi, const long long* pso, int n, const double* occ,
                         const double* w, double* rho_grid, double* rho_w, const long long* rwo) {
  const int k = blockIdx.y;
  const ElemDesc& d = desc[k];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.NE) return;
  const double* pk = Psi + pso[k];
  double r = 0.0, rw = 0.0;
  for (int i = 0; i < n; i++) {
    const double v = pk[(long long)i * d.NE + e];
    r = fma(occ[i] * v, v, r);
    rw = fma(w[i] * v, v, rw);
  }
  rho_w[rwo[k] + e] = rw;
  const int ex = e % d.en[0], ey = (e / d.en[0]) % d.en[1], ez = e / (d.en[0] * d.en[1]);
  // E_k starts at q0 + eo (Q's origin plus E's offset in Q), wrapped into the domain
  const int gx = (d.q0[0] + d.eo[0] + ex) % d.gn[0], gy = (d.q0[1] + d.eo[1] + ey) % d.gn[1],
            gz = (d.q0[2] + d.eo[2] + ez) % d.gn[2];
  atomicAdd(&rho_grid[d.gvoff + ((long long)gz * d.gn[1] + gy) * d.gn[0] + gx], r);
}

__device__ __forceinline__ void gt_dg(double dx, double dy, double dz, double sig, double inv_rc2, double& g,
                                      double& gx, double& gy, double& gz) {
  const double d2 = dx * dx + dy * dy + dz * dz;
  const double one = 1.0 - d2 * inv_rc2;
  if (one <= 0.0) { g = gx = gy = gz = 0.0; return; }
  const double ga = exp(-d2 / (2.0 * sig * sig));
  g = ga * one * one * one;
  const double common = ga * (-(one * one * one) / (sig * sig) - 6.0 * one * one * inv_rc2);
  gx = common * dx; gy = common * dy; gz = common * dz;
}

// Per (element, atom box on E_k): the well term sum_e rho_w dV_I/dR_I dV -> grad_R, and the partial
// overlaps <psi_i, b_l>_{E_k} and <psi_i, db_l/dR_ax>_{E_k} -> pov[atom][16][n] (atomic sums over elements)
__global__ void __launch_bounds__(256) k_dg_atom_terms(const ElemDesc* desc, const AtomBox* boxes,
                                                       const double* dtab, const double* Psi, const long long* pso,
                                                       int n, const double* rho_w, const long long* rwo, double r_cut,
                                                       int npa, double* grad_R, double* pov) {
  const int k = blockIdx.y;
  const ElemDesc& d = desc[k];
  const int bi = blockIdx.x;
  if (bi >= d.pe_count) return;
  const AtomBox& bx = boxes[d.pe_begin + bi];
  __shared__ double cg[kDChunk][4];    // projector g, dg/dd (x, y, z)
  __shared__ int eidx[kDChunk];
  __shared__ double dsp[kDChunk][3];
  const double* t = dtab + bx.toff;
  const int npts = bx.l[0] * bx.l[1] * bx.l[2];
  const double inv_rc2 = 1.0 / (r_cut * r_cut);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const double* pk = Psi + pso[k];
  double fw[3] = {0.0, 0.0, 0.0};
  for (int c0 = 0; c0 < npts; c0 += kDChunk) {
    const int cn = min(kDChunk, npts - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < cn; i += blockDim.x) {
      const int p = c0 + i;
      const int ix = p % bx.l[0], iy = (p / bx.l[0]) % bx.l[1], iz = p / (bx.l[0] * bx.l[1]);
      int ex = bx.s[0] + ix; if (ex >= d.en[0]) ex -= d.en[0];
      int ey = bx.s[1] + iy; if (ey >= d.en[1]) ey -= d.en[1];
      int ez = bx.s[2] + iz; if (ez >= d.en[2]) ez -= d.en[2];
      const double dx = t[ix], dy = t[bx.l[0] + iy], dz = t[bx.l[0] + bx.l[1] + iz];
      const int e = (ez * d.en[1] + ey) * d.en[0] + ex;
      eidx[i] = e;
      dsp[i][0] = dx; dsp[i][1] = dy; dsp[i][2] = dz;
      double g, gx, gy, gz;
      gt_dg(dx, dy, dz, bx.wwidth, inv_rc2, g, gx, gy, gz);
      const double rw = rho_w[rwo[k] + e] * bx.depth * d.dV;
      fw[0] += rw * gx; fw[1] += rw * gy; fw[2] += rw * gz;
      gt_dg(dx, dy, dz, bx.pwidth, inv_rc2, cg[i][0], cg[i][1], cg[i][2], cg[i][3]);
    }
    __syncthreads();
    if (npa == 0) continue;
    // per state (one warp per state): the 16 overlaps of this chunk
    for (int s = warp; s < n; s += nw) {
      const double* ps = pk + (long long)s * d.NE;
      double o[16];
#pragma unroll
      for (int q = 0; q < 16; q++) o[q] = 0.0;
      for (int i = lane; i < cn; i += 32) {
        const double g = cg[i][0];
        if (g == 0.0 && cg[i][1] == 0.0 && cg[i][2] == 0.0 && cg[i][3] == 0.0) continue;
        const double v = ps[eidx[i]] * d.dV;
        const double dg[3] = {cg[i][1], cg[i][2], cg[i][3]};
        // s: b = ns g, db/dR_ax = -ns dg_ax
        o[0] += v * bx.ns * g;
        for (int ax = 0; ax < 3; ax++) o[4 + ax] += -v * bx.ns * dg[ax];
        if (npa == 4) {
          for (int beta = 0; beta < 3; beta++) {
            o[1 + beta] += v * bx.np * dsp[i][beta] * g;
            for (int ax = 0; ax < 3; ax++)
              o[4 + 3 * (1 + beta) + ax] += -v * bx.np * ((beta == ax ? g : 0.0) + dsp[i][beta] * dg[ax]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 16; q++)
        for (int off = 16; off > 0; off >>= 1) o[q] += __shfl_xor_sync(0xffffffffu, o[q], off);
      if (lane < 16) {
        double val = o[0];
#pragma unroll
        for (int q = 1; q < 16; q++) if (lane == q) val = o[q];
        atomicAdd(&pov[((long long)bx.atom * 16 + lane) * n + s], val);
      }
    }
  }
  // well term: block reduction of fw
  __shared__ double red[3][8];
  for (int ax = 0; ax < 3; ax++) {
    double v = fw[ax];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[ax][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int q = 0; q < nw; q++) s += red[threadIdx.x][q];
    atomicAdd(&grad_R[bx.atom * 3 + threadIdx.x], s);
  }
}

// projector term per atom: grad_R[a][ax] += sum_l 2 gamma_l sum_i w_i <psi_i, b_l> <psi_i, db_l/dR_ax>
__global__ void k_dg_force_proj(const double* pov, const double* gamma, int npa, int n, const double* w, int n_atoms,
                                double* grad_R) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_atoms) return;
  const double* pa = pov + (long long)a * 16 * n;
  for (int ax = 0; ax < 3; ax++) {
    double s = 0.0;
    for (int l = 0; l < npa; l++) {
      const double* pb = pa + (long long)l * n;
      const double* pd = pa + (long long)(4 + 3 * l + ax) * n;
      double t = 0.0;
      for (int i = 0; i < n; i++) t += w[i] * pb[i] * pd[i];
      s += 2.0 * gamma[a * npa + l] * t;
    }
    grad_R[a * 3 + ax] += s;
  }
}

}  // namespace
}  // namespace dgdft

using namespace dgdft;

#define DGD_CUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(ctx, DGDFT_CUDA_ERROR, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

#define DGD_WS(ptr, name, bytes)                                                                      \
  do {                                                                                                \
    *(void**)&(ptr) = ws(ctx, name, bytes);                                                           \
    if (!(ptr)) return fail(ctx, DGDFT_OUT_OF_MEMORY, std::string("out of device memory: ") + name);  \
  } while (0)

extern "C" int dgdft_dg_density(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* prm,
                                const dgdft_alb_result* res, const double* eigval, const double* eigvec, int n,
                                double n_electrons, double kT, double* rho, double* energy_mu, double* grad_R,
                                dgdft_stream stream) {
  if (!ctx || !prob || !prm || !res || !res->alb || !eigval || !eigvec || !rho || !energy_mu)
    return fail(ctx, DGDFT_INVALID_ARG, "null argument");
  if (n < 1 || n > kMaxStates) return fail(ctx, DGDFT_INVALID_ARG, "need 1 <= n <= 96 DG states");
  if (!(kT > 0) || !(n_electrons >= 0)) return fail(ctx, DGDFT_INVALID_ARG, "bad kT or electron count");
  if (prm->flags & DGDFT_HOST_BUFFERS) return fail(ctx, DGDFT_UNSUPPORTED, "dgdft_dg_density takes device buffers");
  Plan P;
  std::string msg;
  int r = build_plan(prob, prm, P, msg);
  if (r) return fail(ctx, r, msg);
  cudaStream_t st = (cudaStream_t)stream;
  DGD_CUDA(cudaSetDevice(ctx->device));
  const int M = P.M;
  std::vector<int> h_off(M);
  std::vector<long long> h_pso(M), h_rwo(M);
  long long nb = 0, pso = 0, rwo = 0;
  int max_ne = 0;
  for (int k = 0; k < M; k++) {
    const ElemDesc& d = P.desc[k];
    if (d.n_alb > kMaxStates) return fail(ctx, DGDFT_UNSUPPORTED, "n_alb > 96");
    h_off[k] = int(nb);
    nb += d.n_alb;
    h_pso[k] = pso;
    pso += (long long)n * d.NE;
    h_rwo[k] = rwo;
    rwo += d.NE;
    max_ne = std::max(max_ne, d.NE);
  }
  // device tables: the plan's element descriptors and E boxes, offsets
  ElemDesc* d_desc;
  AtomBox* d_boxes;
  double *d_dtab, *occ, *w, *Psi, *rho_w, *pov, *gam;
  int *d_off, *bad;
  long long *d_pso, *d_rwo;
  DGD_WS(d_desc, "dgd_desc", P.desc.size() * sizeof(ElemDesc));
  DGD_WS(d_boxes, "dgd_boxes", std::max<size_t>(1, P.boxes.size()) * sizeof(AtomBox));
  DGD_WS(d_dtab, "dgd_dtab", P.dtab.size() * sizeof(double));
  DGD_WS(d_off, "dgd_off", M * sizeof(int));
  DGD_WS(d_pso, "dgd_pso", M * sizeof(long long));
  DGD_WS(d_rwo, "dgd_rwo", M * sizeof(long long));
  DGD_WS(occ, "dgd_occ", n * sizeof(double));
  DGD_WS(w, "dgd_w", n * sizeof(double));
  DGD_WS(bad, "dgd_bad", sizeof(int));
  DGD_WS(Psi, "dgd_psi", std::max<long long>(1, pso) * sizeof(double));
  DGD_WS(rho_w, "dgd_rhow", std::max<long long>(1, rwo) * sizeof(double));
  const int npa = prob->n_proj_per_atom;
  const size_t pov_n = size_t(std::max(1, prob->n_atoms)) * 16 * n;
  DGD_WS(pov, "dgd_pov", pov_n * sizeof(double));
  DGD_WS(gam, "dgd_gamma", std::max<size_t>(1, size_t(prob->n_atoms) * std::max(1, npa)) * sizeof(double));
  DGD_CUDA(cudaMemcpyAsync(d_desc, P.desc.data(), P.desc.size() * sizeof(ElemDesc), cudaMemcpyHostToDevice, st));
  if (!P.boxes.empty())
    DGD_CUDA(cudaMemcpyAsync(d_boxes, P.boxes.data(), P.boxes.size() * sizeof(AtomBox), cudaMemcpyHostToDevice, st));
  DGD_CUDA(cudaMemcpyAsync(d_dtab, P.dtab.data(), P.dtab.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  DGD_CUDA(cudaMemcpyAsync(d_off, h_off.data(), M * sizeof(int), cudaMemcpyHostToDevice, st));
  DGD_CUDA(cudaMemcpyAsync(d_pso, h_pso.data(), M * sizeof(long long), cudaMemcpyHostToDevice, st));
  DGD_CUDA(cudaMemcpyAsync(d_rwo, h_rwo.data(), M * sizeof(long long), cudaMemcpyHostToDevice, st));
  if (npa > 0 && prob->n_atoms > 0)
    DGD_CUDA(cudaMemcpyAsync(gam, prob->proj_gamma, size_t(prob->n_atoms) * npa * sizeof(double),
                             cudaMemcpyHostToDevice, st));
  // packed ALB offsets [n_alb][NE] per element (the layout of dgdft_alb_result.alb)
  long long *d_ao;
  DGD_WS(d_ao, "dgd_ao", M * sizeof(long long));
  DGD_CUDA(cudaMemcpyAsync(d_ao, P.off[OFF_A].data(), M * sizeof(long long), cudaMemcpyHostToDevice, st));
  DGD_CUDA(cudaMemsetAsync(rho, 0, P.tot_grid * sizeof(double), st));
  count_launch();
  k_dg_fermi<<<1, 32, 0, st>>>(eigval, n, n_electrons, kT, occ, w, energy_mu, bad);
  const size_t smem = (size_t(n) + kPsiTile) * P.max_nalb * sizeof(double);
  if (smem > 48 * 1024)
    DGD_CUDA(cudaFuncSetAttribute(k_dg_psi, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  count_launch();
  k_dg_psi<<<dim3((max_ne + kPsiTile - 1) / kPsiTile, M), 256, smem, st>>>(d_desc, res->alb, d_ao, eigvec, int(nb), n,
                                                                          d_off, Psi, d_pso);
  count_launch();
  k_dg_rho<<<dim3((max_ne + 255) / 256, M), 256, 0, st>>>(d_desc, Psi, d_pso, n, occ, w, rho, rho_w, d_rwo);
  if (grad_R) {
    DGD_CUDA(cudaMemsetAsync(grad_R, 0, size_t(std::max(1, prob->n_atoms)) * 3 * sizeof(double), st));
    DGD_CUDA(cudaMemsetAsync(pov, 0, pov_n * sizeof(double), st));
    if (P.max_pe > 0) {
      count_launch();
      k_dg_atom_terms<<<dim3(P.max_pe, M), 256, 0, st>>>(d_desc, d_boxes, d_dtab, Psi, d_pso, n, rho_w, d_rwo,
                                                         P.r_cut, npa, grad_R, pov);
    }
    if (npa > 0 && prob->n_atoms > 0) {
      count_launch();
      k_dg_force_proj<<<(prob->n_atoms + 127) / 128, 128, 0, st>>>(pov, gam, npa, n, w, prob->n_atoms, grad_R);
    }
  }
  DGD_CUDA(cudaGetLastError());
  int hbad = 0;
  DGD_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  DGD_CUDA(cudaStreamSynchronize(st));
  if (hbad) return fail(ctx, DGDFT_BAD_INPUT, "the highest DG state is occupied (f >= 1e-12): pass more states");
  return DGDFT_OK;
}
