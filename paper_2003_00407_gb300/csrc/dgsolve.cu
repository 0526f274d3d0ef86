// Eigenpairs of the assembled DG Hamiltonian (Eq. DGEigenvalue: H^DG c = eps c in the orthonormal ALB
// basis) by Chebyshev-filtered subspace iteration (Alg. CheFSI, which the paper applies to H^DG), FP64.
// H^DG is never formed: it is applied from the stencil blocks of dgdft_dg_assemble, block (k, s) coupling
// the test ALBs of element k with the trial ALBs of element neighbors[k][s].  The subspace steps reuse
// the batched dense kernels of the local solve on one "element" whose points are the N_b basis functions.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"
#include "convergence.h"
#include "dgdft.h"
#include "kernels.h"
#include "plan.h"


namespace dgdft {

int fail(dgdft_ctx* c, int code, const std::string& msg);
void* ws(dgdft_ctx* ctx, const std::string& name, size_t bytes);

// Y[v][off_k + i] = sum_s sum_j B[k][s][i][j] X[v][off_n + j]  (n = neighbors[k][s]),
// or, with cheb != null, Y = alpha (H X - c X) + beta Yprev with (alpha, c, beta) = cheb[0..2].
// Block (32, 8): x over the element's rows, y over vectors.
__global__ void k_dg_apply(const double* __restrict__ B, const int* __restrict__ nb, const int* __restrict__ off,
                           const int* __restrict__ nalb, int S, int L, int Nb, int nvec, const double* __restrict__ X,
                           double* __restrict__ Y, const double* __restrict__ Yprev, const double* __restrict__ cheb) {
  const int k = blockIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (v >= nvec) return;
  const int nk = nalb[k];
  const double* xv = X + (long long)v * Nb;
  for (int i = threadIdx.x; i < nk; i += blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < S; s++) {
      const int n = nb[k * S + s];
      if (n < 0) continue;
      const double* row = B + (((long long)k * S + s) * L + i) * L;
      const double* xn = xv + off[n];
      const int nn = nalb[n];
      for (int j = 0; j < nn; j++) acc = fma(row[j], xn[j], acc);
    }
    const long long o = (long long)v * Nb + off[k] + i;
    if (cheb) acc = cheb[0] * (acc - cheb[1] * X[o]) + (Yprev ? cheb[2] * Yprev[o] : 0.0);
    Y[o] = acc;
  }
}

namespace {

struct DGSolve {
  dgdft_ctx* ctx;
  cudaStream_t st;
  int M, S, L, Nb, nblk, nstates, degree, lsteps;   // L: row length of the blocks
  int ld;                                            // leading dimension of the subspace matrices
  const double* B;
  int *nb, *off, *nalb;
  ElemDesc* desc;
  long long *xo, *vo;
  double *X, *Y1, *Y2, *HX, *Lv, *Lf, *Lo;
  double *G1, *G2, *W, *theta, *resid2, *resid, *bounds, *cheb, *alphas, *betas, *ldot, *lmin, *prevres;
  int *flags, *iters, *stall, *active, *hitcap;

  void apply(const double* x, double* y, const double* yprev, const double* ch, int nvec) {
    dim3 grid(M, (nvec + 7) / 8);
    count_launch();
    k_dg_apply<<<grid, dim3(32, 8), 0, st>>>(B, nb, off, nalb, S, L, Nb, nvec, x, y, yprev, ch);
  }
  BatchArgs ba(bool with_flags = true) const { return BatchArgs{desc, with_flags ? flags : nullptr, 1}; }

  // Lanczos upper bound from vector 0 of X (the random start) -> bounds[2]
  void lanczos() {
    BatchArgs b = ba(false);
    launch_convert<double, double>(b, X, xo, Lv, vo, NV_ONE, st);
    cudaMemsetAsync(ldot, 0, sizeof(double), st);
    launch_dot<double>(b, Lv, Lv, vo, ldot, 1, st);
    launch_scale_vec_old<double>(b, Lv, Lv, nullptr, vo, ldot, st);
    cudaMemsetAsync(alphas, 0, lsteps * sizeof(double), st);
    cudaMemsetAsync(betas, 0, lsteps * sizeof(double), st);
    for (int j = 0; j < lsteps; j++) {
      if (j > 0) {
        cudaMemsetAsync(ldot, 0, sizeof(double), st);
        launch_dot<double>(b, Lf, Lf, vo, ldot, 1, st);
        launch_store_sqrt(b, ldot, betas + j, lsteps, st);
        launch_scale_vec_old<double>(b, Lv, Lf, Lo, vo, ldot, st);
      }
      apply(Lv, Lf, nullptr, nullptr, 1);
      launch_dot<double>(b, Lv, Lf, vo, alphas + j, lsteps, st);
      launch_lanczos_update<double>(b, Lv, Lf, Lo, vo, alphas + j, betas + j, lsteps, j == 0, st);
    }
    cudaMemsetAsync(ldot, 0, sizeof(double), st);
    launch_dot<double>(b, Lf, Lf, vo, ldot, 1, st);
    launch_lanczos_bound(b, alphas, betas, lsteps, ldot, bounds, lmin, st);
  }

  void cholqr(double* Yb) {
    BatchArgs b = ba();
    cudaMemsetAsync(G1, 0, size_t(ld) * ld * sizeof(double), st);
    launch_gram<double>(b, Yb, xo, NV_BLK, Yb, xo, NV_BLK, 4, nullptr, nullptr, G1, ld, st);
    launch_chol_inv(b, G1, W, ld, NV_BLK, 1e-13, flags, st);
    launch_rotate<double, double>(b, Yb, xo, Yb, xo, NV_BLK, NV_BLK, 4, W, ld, nullptr, nullptr, nullptr, nullptr, ld,
                                  st);
  }

  // Rayleigh-Ritz of the orthonormalised block Yb: Ritz vectors -> X, H X -> HX, theta, residuals
  void rayleigh_ritz(double* Yb) {
    BatchArgs b = ba();
    apply(Yb, HX, nullptr, nullptr, nblk);
    cudaMemsetAsync(G1, 0, size_t(ld) * ld * sizeof(double), st);
    cudaMemsetAsync(G2, 0, size_t(ld) * ld * sizeof(double), st);
    launch_gram<double>(b, Yb, xo, NV_BLK, Yb, xo, NV_BLK, 4, nullptr, nullptr, G1, ld, st);
    launch_gram<double>(b, Yb, xo, NV_BLK, HX, xo, NV_BLK, 4, nullptr, nullptr, G2, ld, st);
    launch_rr_small(b, G1, G2, W, theta, ld, NV_BLK, flags, st);
    cudaMemsetAsync(resid2, 0, size_t(ld) * sizeof(double), st);
    launch_rotate<double, double>(b, Yb, xo, X, xo, NV_BLK, NV_BLK, 4, W, ld, HX, HX, theta, resid2, ld, st);
  }

  void convergence(double tol) {
    cudaMemsetAsync(active, 0, 4 * sizeof(int), st);
    launch_update_convergence(ba(), resid2, ld, resid, theta, bounds, tol, 0.0, 0, prevres, stall, flags, active,
                              iters, st);
  }
};

}  // namespace
}  // namespace dgdft

using namespace dgdft;

#define DGS_CUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(ctx, DGDFT_CUDA_ERROR, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

#define DGS_WS(ptr, name, bytes)                                                                      \
  do {                                                                                                \
    *(void**)&(ptr) = ws(ctx, name, bytes);                                                           \
    if (!(ptr)) return fail(ctx, DGDFT_OUT_OF_MEMORY, std::string("out of device memory: ") + name);  \
  } while (0)

extern "C" int dgdft_dg_eigensolve(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* prm,
                                   const double* blocks, const dgdft_dg_solve_params* sp, double* eigval,
                                   double* resid, double* eigvec, int* iters, dgdft_stream stream) {
  if (!ctx || !prob || !prm || !blocks || !sp || !eigval || !resid || !iters)
    return fail(ctx, DGDFT_INVALID_ARG, "null argument");
  Plan P;
  std::string msg;
  int r = build_plan(prob, prm, P, msg);
  if (r) return fail(ctx, r, msg);
  DGSolve d{};
  d.ctx = ctx;
  d.st = (cudaStream_t)stream;
  d.M = P.M;
  d.S = P.n_stencil;
  d.L = P.L;
  std::vector<int> h_off(P.M), h_nalb(P.M), h_nb(size_t(P.M) * P.n_stencil);
  long long nb_tot = 0;
  for (int k = 0; k < P.M; k++) {
    h_off[k] = int(nb_tot);
    h_nalb[k] = P.desc[k].n_alb;
    nb_tot += P.desc[k].n_alb;
    for (int s = 0; s < P.n_stencil; s++)
      h_nb[size_t(k) * P.n_stencil + s] = P.n_stencil > 1 ? prob->neighbors[k * P.n_stencil + s] : k;
  }
  if (nb_tot >= (1LL << 24)) return fail(ctx, DGDFT_UNSUPPORTED, "more than 2^24 basis functions");
  d.Nb = int(nb_tot);
  d.nblk = sp->n_blk;
  d.nstates = sp->n_states;
  d.degree = sp->cheb_degree;
  d.lsteps = sp->lanczos_steps > 0 ? sp->lanczos_steps : 10;
  d.ld = std::max(sp->n_blk, 1);
  if (d.nstates < 1 || d.nblk < d.nstates || d.nblk > 96 || d.nblk > d.Nb)
    return fail(ctx, DGDFT_INVALID_ARG, "need 1 <= n_states <= n_blk <= min(96, N_b)");
  if (d.degree < 2 || sp->max_iter < 0 || !(sp->tol > 0)) return fail(ctx, DGDFT_INVALID_ARG, "bad degree, max_iter or tol");
  const bool host = (prm->flags & DGDFT_HOST_BUFFERS) != 0;
  cudaStream_t st = d.st;
  DGS_CUDA(cudaSetDevice(ctx->device));
  const size_t L = std::max(d.nblk, 1), blk = size_t(d.nblk) * d.Nb;
  // inputs
  d.B = blocks;
  const size_t bsz = size_t(P.M) * P.n_stencil * P.L * P.L;
  if (host) {
    double* dB;
    DGS_WS(dB, "dgs_blocks", bsz * sizeof(double));
    DGS_CUDA(cudaMemcpyAsync(dB, blocks, bsz * sizeof(double), cudaMemcpyHostToDevice, st));
    d.B = dB;
  }
  DGS_WS(d.nb, "dgs_nb", h_nb.size() * sizeof(int));
  DGS_WS(d.off, "dgs_off", h_off.size() * sizeof(int));
  DGS_WS(d.nalb, "dgs_nalb", h_nalb.size() * sizeof(int));
  DGS_CUDA(cudaMemcpyAsync(d.nb, h_nb.data(), h_nb.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  DGS_CUDA(cudaMemcpyAsync(d.off, h_off.data(), h_off.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  DGS_CUDA(cudaMemcpyAsync(d.nalb, h_nalb.data(), h_nalb.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  // one element of N_b points carries the subspace steps
  ElemDesc e{};
  e.N = e.NE = d.Nb;
  e.n_blk = d.nblk;
  e.n_eig = e.n_alb = d.nstates;
  e.dV = 1.0;
  e.qn[0] = e.en[0] = d.Nb;
  e.qn[1] = e.qn[2] = e.en[1] = e.en[2] = 1;
  const long long zero = 0;
  DGS_WS(d.desc, "dgs_desc", sizeof(ElemDesc));
  DGS_WS(d.xo, "dgs_xo", sizeof(long long));
  DGS_WS(d.vo, "dgs_vo", sizeof(long long));
  DGS_CUDA(cudaMemcpyAsync(d.desc, &e, sizeof(ElemDesc), cudaMemcpyHostToDevice, st));
  DGS_CUDA(cudaMemcpyAsync(d.xo, &zero, sizeof(long long), cudaMemcpyHostToDevice, st));
  DGS_CUDA(cudaMemcpyAsync(d.vo, &zero, sizeof(long long), cudaMemcpyHostToDevice, st));
  DGS_WS(d.X, "dgs_X", blk * sizeof(double));
  DGS_WS(d.Y1, "dgs_Y1", blk * sizeof(double));
  DGS_WS(d.Y2, "dgs_Y2", blk * sizeof(double));
  DGS_WS(d.HX, "dgs_HX", blk * sizeof(double));
  DGS_WS(d.Lv, "dgs_Lv", size_t(d.Nb) * sizeof(double));
  DGS_WS(d.Lf, "dgs_Lf", size_t(d.Nb) * sizeof(double));
  DGS_WS(d.Lo, "dgs_Lo", size_t(d.Nb) * sizeof(double));
  DGS_WS(d.G1, "dgs_G1", L * L * sizeof(double));
  DGS_WS(d.G2, "dgs_G2", L * L * sizeof(double));
  DGS_WS(d.W, "dgs_W", L * L * sizeof(double));
  DGS_WS(d.theta, "dgs_theta", L * sizeof(double));
  DGS_WS(d.resid2, "dgs_resid2", L * sizeof(double));
  DGS_WS(d.resid, "dgs_resid", L * sizeof(double));
  DGS_WS(d.bounds, "dgs_bounds", 3 * sizeof(double));
  DGS_WS(d.cheb, "dgs_cheb", 3 * size_t(d.degree) * sizeof(double));
  DGS_WS(d.alphas, "dgs_alphas", d.lsteps * sizeof(double));
  DGS_WS(d.betas, "dgs_betas", d.lsteps * sizeof(double));
  DGS_WS(d.ldot, "dgs_ldot", sizeof(double));
  DGS_WS(d.lmin, "dgs_lmin", sizeof(double));
  DGS_WS(d.prevres, "dgs_prevres", sizeof(double));
  DGS_WS(d.flags, "dgs_flags", sizeof(int));
  DGS_WS(d.iters, "dgs_iters", sizeof(int));
  DGS_WS(d.stall, "dgs_stall", sizeof(int));
  DGS_WS(d.active, "dgs_active", 4 * sizeof(int));
  d.hitcap = nullptr;
  int* h_active = nullptr;
  DGS_CUDA(cudaMallocHost(&h_active, 4 * sizeof(int)));
  struct FreeHost {
    int* p;
    ~FreeHost() { cudaFreeHost(p); }
  } fh{h_active};
  g_max_points = d.Nb;
  g_max_nblk = d.nblk;
  g_max_nalb = d.nstates;
  const double big = 1e300;
  DGS_CUDA(cudaMemsetAsync(d.flags, 0, sizeof(int), st));
  DGS_CUDA(cudaMemsetAsync(d.iters, 0xFF, sizeof(int), st));
  DGS_CUDA(cudaMemsetAsync(d.stall, 0, sizeof(int), st));
  DGS_CUDA(cudaMemsetAsync(d.bounds, 0, 3 * sizeof(double), st));
  DGS_CUDA(cudaMemcpyAsync(d.prevres, &big, sizeof(double), cudaMemcpyHostToDevice, st));
  BatchArgs b1{d.desc, nullptr, 1};
  launch_set_active(b1, d.flags, st);
  // SplitMix64 start (element 0), Lanczos bound, CholQR2, start-up Rayleigh-Ritz
  launch_random_init<double>(b1, d.X, d.xo, sp->seed, st);
  d.lanczos();
  d.cholqr(d.X);
  d.cholqr(d.X);
  DGS_CUDA(cudaMemcpyAsync(d.Y1, d.X, blk * sizeof(double), cudaMemcpyDeviceToDevice, st));
  d.rayleigh_ritz(d.Y1);
  d.convergence(sp->tol);
  int passes_done = 0;
  bool capped = false;
  for (int it = 0;; it++) {
    DGS_CUDA(cudaMemcpyAsync(h_active, d.active, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    DGS_CUDA(cudaStreamSynchronize(st));
    if (h_active[0] == 0) break;
    if (it == sp->max_iter) {
      capped = true;
      break;
    }
    // filter: Y1 = p_1(H) X, then the three-term recurrence over Y1, Y2 and HX as the spare
    launch_cheb_coeffs(b1, d.bounds, d.cheb, d.degree, st);
    d.apply(d.X, d.Y1, nullptr, d.cheb, d.nblk);        // (alpha, c, beta = 0) of step 1
    double* prev = d.X;
    double* cur = d.Y1;
    double* spare = d.Y2;
    for (int step = 1; step < d.degree; step++) {
      d.apply(cur, spare, prev, d.cheb + 3 * step, d.nblk);
      double* t = prev;
      prev = cur;
      cur = spare;
      spare = (t == d.X) ? d.HX : t;   // X is read by the first step only; HX is free until the RR
    }
    if (cur != d.Y1) DGS_CUDA(cudaMemcpyAsync(d.Y1, cur, blk * sizeof(double), cudaMemcpyDeviceToDevice, st));
    d.cholqr(d.Y1);
    d.cholqr(d.Y1);
    d.rayleigh_ritz(d.Y1);
    d.convergence(sp->tol);
    passes_done++;
  }
  DGS_CUDA(cudaGetLastError());
  // outputs
  double *o_ev = eigval, *o_res = resid, *o_vec = eigvec;
  int* o_it = iters;
  if (host) {
    DGS_WS(o_ev, "dgs_o_ev", L * sizeof(double));
    DGS_WS(o_res, "dgs_o_res", L * sizeof(double));
    DGS_WS(o_it, "dgs_o_it", sizeof(int));
    if (eigvec) DGS_WS(o_vec, "dgs_o_vec", blk * sizeof(double));
  }
  DGS_CUDA(cudaMemcpyAsync(o_ev, d.theta, d.nblk * sizeof(double), cudaMemcpyDeviceToDevice, st));
  DGS_CUDA(cudaMemcpyAsync(o_res, d.resid, d.nblk * sizeof(double), cudaMemcpyDeviceToDevice, st));
  DGS_CUDA(cudaMemcpyAsync(o_it, d.iters, sizeof(int), cudaMemcpyDeviceToDevice, st));
  if (eigvec) DGS_CUDA(cudaMemcpyAsync(o_vec, d.X, blk * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (host) {
    DGS_CUDA(cudaMemcpyAsync(eigval, o_ev, d.nblk * sizeof(double), cudaMemcpyDeviceToHost, st));
    DGS_CUDA(cudaMemcpyAsync(resid, o_res, d.nblk * sizeof(double), cudaMemcpyDeviceToHost, st));
    DGS_CUDA(cudaMemcpyAsync(iters, o_it, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (eigvec) DGS_CUDA(cudaMemcpyAsync(eigvec, o_vec, blk * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  int hflags = 0;
  DGS_CUDA(cudaMemcpyAsync(h_active, d.flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  DGS_CUDA(cudaStreamSynchronize(st));
  hflags = h_active[0];
  (void)passes_done;
  if (hflags & EF_BAD) return fail(ctx, DGDFT_BAD_INPUT, "non-finite residual in the DG eigensolve");
  if (hflags & EF_CHOL_FAIL) return fail(ctx, DGDFT_CHOLESKY_FAIL, "Cholesky-QR failed in the DG eigensolve");
  if (capped) return fail(ctx, DGDFT_NOT_CONVERGED, "DG eigensolve reached max_iter");
  return DGDFT_OK;
}
