// C-ABI of libdgdft: argument checks, per-call planning (element descriptors,
// atom boxes, shape groups, packed offsets), the device workspace, and the
// CheFSI driver (Alg. CheFSI) behind dgdft_alb_generate.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "dgdft.h"
#include "convergence.h"
#include "kernels.h"
#include "plan.h"

#include "context.h"

namespace dgdft {

long long g_launches = 0;

static thread_local std::string g_last_error;  // for failures without a context

int fail(dgdft_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  g_last_error = msg;
  return code;
}

#define CUDA_OK(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(ctx, DGDFT_CUDA_ERROR, std::string(#call) + ": " + cudaGetErrorString(e_));  \
  } while (0)

// grow-only named device buffers
void* ws(dgdft_ctx* ctx, const std::string& name, size_t bytes) {
  if (bytes == 0) bytes = 16;
  auto it = ctx->bufs.find(name);
  if (it != ctx->bufs.end()) {
    if (it->second.second >= bytes) return it->second.first;
    cudaFree(it->second.first);
    ctx->bufs.erase(it);
  }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  ctx->bufs[name] = {p, bytes};
  return p;
}

int init_twiddles(dgdft_ctx* ctx) {
  if (ctx->tw_ready) return DGDFT_OK;
  std::vector<double2> t64(kTwiddleCount);
  std::vector<float2> t32(kTwiddleCount);
  for (int n = 1; n <= kMaxLine; n++)
    for (int m = 0; m < n; m++) {
      const double a = -2.0 * M_PI * double(m) / double(n);
      t64[twiddle_offset(n) + m] = make_double2(std::cos(a), std::sin(a));
      t32[twiddle_offset(n) + m] = make_float2(float(std::cos(a)), float(std::sin(a)));
    }
  if (upload_twiddles(t64.data(), t32.data()) || upload_fused_twiddles(t32.data()))
    return fail(ctx, DGDFT_CUDA_ERROR, "twiddle upload failed");
  if (set_hx_smem_limits() || set_linalg_smem_limits() || set_fused_smem_limits()) {
    cudaGetLastError();
    return fail(ctx, DGDFT_CUDA_ERROR, "cudaFuncSetAttribute(max dynamic shared memory) failed");
  }
  ctx->tw_ready = true;
  return DGDFT_OK;
}

template <typename T> struct Typed {};

// ---------------------------------------------------------------------------
// Upload the plan's device tables (desc, boxes, offsets, group lists).
int upload_plan(dgdft_ctx* ctx, Plan& P, cudaStream_t st) {
  auto up = [&](const std::string& name, const void* src, size_t bytes, void** dst) -> int {
    *dst = ws(ctx, name, bytes);
    if (!*dst) return fail(ctx, DGDFT_OUT_OF_MEMORY, "workspace allocation failed: " + name);
    if (bytes) {
      cudaError_t e = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return fail(ctx, DGDFT_CUDA_ERROR, cudaGetErrorString(e));
    }
    return DGDFT_OK;
  };
  int r;
  if ((r = up("p_desc", P.desc.data(), P.desc.size() * sizeof(ElemDesc), (void**)&P.d_desc))) return r;
  if ((r = up("p_boxes", P.boxes.data(), P.boxes.size() * sizeof(AtomBox), (void**)&P.d_boxes))) return r;
  if ((r = up("p_dtab", P.dtab.data(), P.dtab.size() * sizeof(double), (void**)&P.d_dtab))) return r;
  if ((r = up("p_fatoms", P.fatoms.data(), std::max<size_t>(1, P.fatoms.size()) * sizeof(FusedAtomRec),
              (void**)&P.d_fatoms)))
    return r;
  {
    // compact projector-point lists of the Q boxes (read by the fused kernel)
    const size_t nq = size_t(std::max(1, P.n_qboxes));
    P.plist.gw = (uint2*)ws(ctx, "p_plist_gw", nq * kProjCap * sizeof(uint2));
    P.plist.n = (int*)ws(ctx, "p_plist_n", 2 * nq * sizeof(int));
    if (!P.plist.gw || !P.plist.n) return fail(ctx, DGDFT_OUT_OF_MEMORY, "workspace allocation failed: p_plist");
    if (P.n_qboxes > 0) launch_build_proj_lists(P.d_fatoms, P.d_dtab, P.n_qboxes, P.r_cut, P.plist, st);
  }
  const char* names[kOffKinds] = {"p_ox", "p_oe", "p_oa", "p_ov", "p_os", "p_ofe", "p_ove"};
  for (int i = 0; i < kOffKinds; i++)
    if ((r = up(names[i], P.off[i].data(), P.off[i].size() * sizeof(long long), (void**)&P.d_off[i]))) return r;
  for (size_t g = 0; g < P.hx.groups.size(); g++) {
    ShapeGroup& G = P.hx.groups[g];
    if ((r = up("p_grp" + std::to_string(g), G.elems.data(), G.elems.size() * sizeof(int), (void**)&G.d_elems)))
      return r;
  }
  g_max_points = P.max_points;
  g_max_nblk = P.max_nblk;
  g_max_nalb = P.max_nalb;
  return DGDFT_OK;
}

HxArgs hx_args(const Plan& P, const int* flags, int kind, int nvec_mode) {
  HxArgs a;
  a.desc = P.d_desc;
  a.elems = nullptr;
  a.flags = flags;
  a.boxes = P.d_boxes;
  a.dtab = P.d_dtab;
  a.xo = P.d_off[kind];
  a.so = P.d_off[OFF_S];
  a.nvec_mode = nvec_mode;
  a.n_proj_per_atom = P.n_proj_per_atom;
  a.r_cut = P.r_cut;
  a.fatoms = P.d_fatoms;
  a.plist = P.plist;
  return a;
}

void set_group_nvec(Plan& P, int mode) {
  for (auto& g : P.hx.groups)
    g.max_nvec = mode == NV_BLK ? g.max_nblk : (mode == NV_EIG ? g.max_neig : (mode == NV_ALB ? g.max_nalb : 1));
}

// ---------------------------------------------------------------------------
// Work buffers of one precision stage.
template <typename T> struct Stage {
  T *B[3], *HY, *Lv, *Lf, *Lvold;
  cplx<T>* S;
};

struct Common {
  double *V64, *bounds, *cheb, *G1, *G2, *W, *theta, *resid2, *resid, *P, *prevres, *alphas, *betas, *ldot, *lmin;
  float* V32;
  int *flags, *iters, *stall, *active, *hitcap, *pdeg;
};

#define WS(ptr, name, bytes)                                                             \
  do {                                                                                   \
    *(void**)&(ptr) = ws(ctx, name, bytes);                                              \
    if (!(ptr)) return fail(ctx, DGDFT_OUT_OF_MEMORY, std::string("out of device memory: ") + name); \
  } while (0)

// All [n_blk][N] block buffers live in one arena, in units of one FP32 block
// set (u = 4 * tot_x bytes), reused across stages:
//   mixed FP32 stage : B0 [0,1) B1 [1,2) B2 [2,3) HY [3,4)
//   mixed FP64 sweep : X64 [4,6) (promoted from B0) and HX64 [1,3)
//   FP64 path        : B0 [0,2) B1 [2,4) B2 [4,6) HY [6,8)
//   DG assembly      : psi [0,2) and derivatives [2,4)  (n_alb <= n_blk rows)
char* arena(dgdft_ctx* ctx, const Plan& P, int units) {
  return (char*)ws(ctx, "arena", size_t(units) * size_t(P.tot[OFF_X]) * 4);
}

template <typename T>
int stage_lanczos(dgdft_ctx* ctx, const Plan& P, Stage<T>& s) {
  const char* sfx = sizeof(T) == 4 ? "32" : "64";
  WS(s.S, "S_spec", size_t(P.tot[OFF_S]) * sizeof(cplx<double>));  // shared by both precisions
  WS(s.Lv, std::string("Lv_") + sfx, size_t(P.tot[OFF_V]) * sizeof(T));
  WS(s.Lf, std::string("Lf_") + sfx, size_t(P.tot[OFF_V]) * sizeof(T));
  WS(s.Lvold, std::string("Lo_") + sfx, size_t(P.tot[OFF_V]) * sizeof(T));
  return DGDFT_OK;
}

// Stage whose four blocks start at arena units u0..u3 (each block sizeof(T)/4 units)
template <typename T>
int get_stage(dgdft_ctx* ctx, const Plan& P, Stage<T>& s, int units, const int u[4]) {
  char* ar = arena(ctx, P, units);
  if (!ar) return fail(ctx, DGDFT_OUT_OF_MEMORY, "out of device memory: block arena");
  const size_t unit = size_t(P.tot[OFF_X]) * 4;
  s.B[0] = (T*)(ar + u[0] * unit);
  s.B[1] = (T*)(ar + u[1] * unit);
  s.B[2] = (T*)(ar + u[2] * unit);
  s.HY = (T*)(ar + u[3] * unit);
  return stage_lanczos<T>(ctx, P, s);
}

int get_common(dgdft_ctx* ctx, const Plan& P, int degree, int lsteps, Common& c) {
  const size_t M = P.M, L = P.L;
  WS(c.V64, "V64", P.tot[OFF_V] * sizeof(double));
  WS(c.V32, "V32", P.tot[OFF_V] * sizeof(float));
  WS(c.bounds, "bounds", M * 3 * sizeof(double));
  WS(c.cheb, "cheb", M * 3 * degree * sizeof(double));
  WS(c.G1, "G1", M * L * L * sizeof(double));
  WS(c.G2, "G2", M * L * L * sizeof(double));
  WS(c.W, "W", M * L * L * sizeof(double));
  WS(c.theta, "theta", M * L * sizeof(double));
  WS(c.resid2, "resid2", M * L * sizeof(double));
  WS(c.resid, "resid", M * L * sizeof(double));
  WS(c.P, "Pproj", std::max<size_t>(1, P.tot_p) * sizeof(double));
  WS(c.prevres, "prevres", M * sizeof(double));
  WS(c.alphas, "alphas", M * lsteps * sizeof(double));
  WS(c.betas, "betas", M * lsteps * sizeof(double));
  WS(c.ldot, "ldot", M * sizeof(double));
  WS(c.lmin, "lmin", M * sizeof(double));
  WS(c.flags, "flags", M * sizeof(int));
  WS(c.iters, "iters", M * sizeof(int));
  WS(c.stall, "stall", M * sizeof(int));
  WS(c.active, "active", 4 * sizeof(int));   // [0] active count, [2..3] max residual (double bits)
  WS(c.hitcap, "hitcap", M * sizeof(int));
  WS(c.pdeg, "pdeg", M * sizeof(int));
  return DGDFT_OK;
}

// H X (apply) or a Chebyshev step, with projections recomputed for X
template <typename T>
void hx(Plan& P, const Common& c, const int* flags, int kind, int nvmode, const T* X, T* Y, const T* Yprev,
        cplx<T>* S, const double* cheb, int cheb_stride, int out_mode, cudaStream_t st);

template <typename T> const T* vq(const Common& c);
template <> const float* vq<float>(const Common& c) { return c.V32; }
template <> const double* vq<double>(const Common& c) { return c.V64; }

template <typename T>
void hx(Plan& P, const Common& c, const int* flags, int kind, int nvmode, const T* X, T* Y, const T* Yprev,
        cplx<T>* S, const double* cheb, int cheb_stride, int out_mode, cudaStream_t st) {
  if (P.tot_p > 0) cudaMemsetAsync(c.P, 0, P.tot_p * sizeof(double), st);
  set_group_nvec(P, nvmode);
  HxArgs a = hx_args(P, flags, kind, nvmode);
  launch_hx<T>(P.hx, a, X, Y, Yprev, vq<T>(c), S, P.tot_p > 0 ? c.P : nullptr, cheb, cheb_stride, out_mode,
               MULT_KINETIC, st);
}

// Lanczos upper bound b_up from vector 0 of the block in B[0] -> bounds[k][2]
template <typename T>
void lanczos(Plan& P, const Common& c, Stage<T>& s, int steps, cudaStream_t st) {
  BatchArgs b{P.d_desc, nullptr, P.M};
  const long long* ov = P.d_off[OFF_V];
  launch_convert<T, T>(b, s.B[0], P.d_off[OFF_X], s.Lv, ov, NV_ONE, st);
  cudaMemsetAsync(c.ldot, 0, P.M * sizeof(double), st);
  launch_dot<T>(b, s.Lv, s.Lv, ov, c.ldot, 1, st);
  launch_scale_vec_old<T>(b, s.Lv, s.Lv, nullptr, ov, c.ldot, st);
  cudaMemsetAsync(c.alphas, 0, P.M * steps * sizeof(double), st);
  cudaMemsetAsync(c.betas, 0, P.M * steps * sizeof(double), st);
  for (int j = 0; j < steps; j++) {
    if (j > 0) {
      cudaMemsetAsync(c.ldot, 0, P.M * sizeof(double), st);
      launch_dot<T>(b, s.Lf, s.Lf, ov, c.ldot, 1, st);
      launch_store_sqrt(b, c.ldot, c.betas + j, steps, st);
      launch_scale_vec_old<T>(b, s.Lv, s.Lf, s.Lvold, ov, c.ldot, st);
    }
    hx<T>(P, c, nullptr, OFF_V, NV_ONE, s.Lv, s.Lf, nullptr, s.S, nullptr, 0, OUT_APPLY, st);
    launch_dot<T>(b, s.Lv, s.Lf, ov, c.alphas + j, steps, st);
    launch_lanczos_update<T>(b, s.Lv, s.Lf, s.Lvold, ov, c.alphas + j, c.betas + j, steps, j == 0, st);
  }
  cudaMemsetAsync(c.ldot, 0, P.M * sizeof(double), st);
  launch_dot<T>(b, s.Lf, s.Lf, ov, c.ldot, 1, st);
  launch_lanczos_bound(b, c.alphas, c.betas, steps, c.ldot, c.bounds, c.lmin, st);
}

// Rayleigh-Ritz of the orthonormalised block Y: X -> B[0], HX -> HY, theta, residuals
template <typename T>
void rayleigh_ritz(Plan& P, const Common& c, Stage<T>& s, T* Y, cudaStream_t st) {
  BatchArgs b{P.d_desc, c.flags, P.M};
  const long long* ox = P.d_off[OFF_X];
  const size_t mat = size_t(P.M) * P.L * P.L * sizeof(double);
  hx<T>(P, c, c.flags, OFF_X, NV_BLK, Y, s.HY, nullptr, s.S, nullptr, 0, OUT_APPLY, st);
  cudaMemsetAsync(c.G1, 0, mat, st);
  cudaMemsetAsync(c.G2, 0, mat, st);
  launch_gram<T>(b, Y, ox, NV_BLK, Y, ox, NV_BLK, 4, nullptr, nullptr, c.G1, P.L, st);
  launch_gram<T>(b, Y, ox, NV_BLK, s.HY, ox, NV_BLK, 4, nullptr, nullptr, c.G2, P.L, st);
  launch_rr_small(b, c.G1, c.G2, c.W, c.theta, P.L, NV_BLK, c.flags, st);
  cudaMemsetAsync(c.resid2, 0, size_t(P.M) * P.L * sizeof(double), st);
  launch_rotate<T, T>(b, Y, ox, s.B[0], ox, NV_BLK, NV_BLK, 4, c.W, P.L, s.HY, s.HY, c.theta, c.resid2, P.L, st);
}

template <typename T>
void cholqr(Plan& P, const Common& c, T* Y, double rel_shift, cudaStream_t st) {
  BatchArgs b{P.d_desc, c.flags, P.M};
  const long long* ox = P.d_off[OFF_X];
  cudaMemsetAsync(c.G1, 0, size_t(P.M) * P.L * P.L * sizeof(double), st);
  launch_gram<T>(b, Y, ox, NV_BLK, Y, ox, NV_BLK, 4, nullptr, nullptr, c.G1, P.L, st);
  launch_chol_inv(b, c.G1, c.W, P.L, NV_BLK, rel_shift, c.flags, st);
  launch_rotate<T, T>(b, Y, ox, Y, ox, NV_BLK, NV_BLK, 4, c.W, P.L, nullptr, nullptr, nullptr, nullptr, P.L, st);
}

// One precision stage of CheFSI.  On entry B[0] holds the random start block; a warm start x0
// ([n_eig][N] per element, eigvec layout) replaces its first n_eig vectors after the Lanczos bound,
// which keeps its random vector 0 (a Lanczos run started from an eigenvector stops at once and
// would give no bound).  On exit B[0] holds the Ritz vectors of every element.
template <typename T>
int chefsi_stage(dgdft_ctx* ctx, Plan& P, const Common& c, Stage<T>& s, const dgdft_alb_params* prm, int degree,
                 int lsteps, bool mixed, cudaStream_t st, double* history, const double* x0) {
  if (history)
    for (int i = 0; i < prm->max_iter + 2; i++) history[i] = -1.0;
  BatchArgs b{P.d_desc, c.flags, P.M};
  const double rel_shift = sizeof(T) == 4 ? 1e-6 : 1e-13;
  lanczos<T>(P, c, s, lsteps, st);
  if (x0) {
    BatchArgs ball{P.d_desc, nullptr, P.M};
    launch_convert<double, T>(ball, x0, P.d_off[OFF_E], s.B[0], P.d_off[OFF_X], NV_EIG, st);
  }
  cholqr<T>(P, c, s.B[0], rel_shift, st);
  cholqr<T>(P, c, s.B[0], rel_shift, st);
  rayleigh_ritz<T>(P, c, s, s.B[0], st);
  const double tol_mixed = prm->tol_mixed > 0 ? prm->tol_mixed : 1e-6;
  cudaMemsetAsync(c.active, 0, 4 * sizeof(int), st);
  launch_update_convergence(b, c.resid2, P.L, c.resid, c.theta, c.bounds, prm->tol, tol_mixed, mixed ? 1 : 0,
                            c.prevres, c.stall, c.flags, c.active, c.iters, st);
  launch_first_a0(b, c.lmin, c.bounds, st);
  // filter degree per pass and element (a reading of the paper's fixed m): the requested degree on the first
  // pass (a random block has no converged Ritz vectors to keep), then at most what the precision carries
  // over the element's spectrum: growth cosh(m acosh|x(a0)|) <= 1e10 in FP32, 1e15 in FP64; the pass runs
  // the largest of these and elements with a smaller one stop early
  const double range_log = sizeof(T) == 4 ? 23.72 : 35.23;
  launch_pass_degree(b, c.bounds, degree, 1e300, c.pdeg, c.active + 1, st);
  // the start Rayleigh-Ritz is not a filter pass
  for (int it = 0; it <= prm->max_iter; it++) {
    CUDA_OK(cudaMemcpyAsync(ctx->h_active, c.active, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaStreamSynchronize(st));
    const int deg = std::max(2, std::min(degree, ctx->h_active[1]));
    if (history) {
      double mx;
      std::memcpy(&mx, ctx->h_active + 2, sizeof(double));
      history[it] = mx;
    }
    if (*ctx->h_active == 0) break;
    if (it == prm->max_iter) {
      // elements still active hit the cap
      std::vector<int> hf(P.M);
      CUDA_OK(cudaMemcpy(hf.data(), c.flags, P.M * sizeof(int), cudaMemcpyDeviceToHost));
      std::vector<int> hc(P.M, 0);
      for (int k = 0; k < P.M; k++) hc[k] = (hf[k] & EF_ACTIVE) ? 1 : 0;
      CUDA_OK(cudaMemcpy(c.hitcap, hc.data(), P.M * sizeof(int), cudaMemcpyHostToDevice));
      break;
    }
    launch_cheb_coeffs(b, c.bounds, c.cheb, deg, st, c.pdeg);
    launch_cheb_first<T>(b, s.B[0], s.HY, s.B[1], P.d_off[OFF_X], c.cheb, 3 * deg, st);
    T* prev = s.B[0];
    T* cur = s.B[1];
    T* spare = s.B[2];
    for (int step = 1; step < deg; step++) {
      hx<T>(P, c, c.flags, OFF_X, NV_BLK, cur, spare, prev, s.S, c.cheb + 3 * step, 3 * deg, OUT_CHEB, st);
      T* t = prev;
      prev = cur;
      cur = spare;
      spare = t;
    }
    cholqr<T>(P, c, cur, rel_shift, st);
    rayleigh_ritz<T>(P, c, s, cur, st);
    cudaMemsetAsync(c.active, 0, 4 * sizeof(int), st);
    launch_update_convergence(b, c.resid2, P.L, c.resid, c.theta, c.bounds, prm->tol, tol_mixed, mixed ? 1 : 0,
                              c.prevres, c.stall, c.flags, c.active, c.iters, st);
    launch_pass_degree(b, c.bounds, degree, range_log, c.pdeg, c.active + 1, st);
  }
  CUDA_OK(cudaGetLastError());
  return DGDFT_OK;
}

// LOBPCG local solver with the Teter preconditioner (Alg. LOBPCG, Eqs. 3-5), FP64, the same block size n
// (<= 32) in every element.  On entry X holds the random start; on exit X holds the Ritz vectors, c.theta /
// c.resid the Ritz values and residuals (ld P.L) and c.iters the iteration count.  The projected problem
// over [X, W, P] (3n <= 96) is solved by the generalised Rayleigh-Ritz kernel of the CheFSI path.
int lobpcg_stage(dgdft_ctx* ctx, Plan& P, const Common& c, const dgdft_alb_params* prm, double* X,
                 cudaStream_t st, double* history, double** x_out) {
  if (history)
    for (int i = 0; i < prm->max_iter + 2; i++) history[i] = -1.0;
  const int M = P.M, n = P.desc.empty() ? 0 : P.desc[0].n_blk;
  const int L3 = 3 * P.L;
  const size_t blk = size_t(P.tot[OFF_X]) * sizeof(double);
  double *HX, *W, *HW, *Pd, *HP, *Xn, *HXn, *Pn, *HPn, *TX, *C3, *G3, *A3, *th3, *r3, *rs3, *ek;
  cplx<double>* S;
  WS(HX, "lob_HX", blk);
  WS(W, "lob_W", blk);
  WS(HW, "lob_HW", blk);
  WS(Pd, "lob_P", blk);
  WS(HP, "lob_HP", blk);
  WS(Xn, "lob_Xn", blk);
  WS(HXn, "lob_HXn", blk);
  WS(Pn, "lob_Pn", blk);
  WS(HPn, "lob_HPn", blk);
  WS(TX, "lob_TX", blk);
  WS(S, "S_spec", size_t(P.tot[OFF_S]) * sizeof(cplx<double>));
  WS(C3, "lob_C3", size_t(M) * L3 * L3 * sizeof(double));
  WS(G3, "lob_G3", size_t(M) * L3 * L3 * sizeof(double));
  WS(A3, "lob_A3", size_t(M) * L3 * L3 * sizeof(double));
  WS(th3, "lob_theta", size_t(M) * L3 * sizeof(double));
  WS(r3, "lob_resid2", size_t(M) * L3 * sizeof(double));
  WS(rs3, "lob_resid", size_t(M) * L3 * sizeof(double));
  WS(ek, "lob_ekin", size_t(M) * L3 * sizeof(double));
  // element descriptors with the trial-subspace sizes 2n and 3n for the projected problem
  ElemDesc *d2, *d3;
  WS(d2, "lob_desc2", size_t(M) * sizeof(ElemDesc));
  WS(d3, "lob_desc3", size_t(M) * sizeof(ElemDesc));
  {
    std::vector<ElemDesc> h2(P.desc), h3(P.desc);
    for (int k = 0; k < M; k++) {
      h2[k].n_blk = 2 * n;
      h3[k].n_blk = 3 * n;
    }
    CUDA_OK(cudaMemcpyAsync(d2, h2.data(), M * sizeof(ElemDesc), cudaMemcpyHostToDevice, st));
    CUDA_OK(cudaMemcpyAsync(d3, h3.data(), M * sizeof(ElemDesc), cudaMemcpyHostToDevice, st));
    CUDA_OK(cudaStreamSynchronize(st));   // h2, h3 are host temporaries
  }
  BatchArgs b{P.d_desc, c.flags, M};
  const long long* ox = P.d_off[OFF_X];
  const size_t mat3 = size_t(M) * L3 * L3 * sizeof(double);
  HxArgs ha = hx_args(P, c.flags, OFF_X, NV_BLK);
  set_group_nvec(P, NV_BLK);
  // start: CholQR2 and Rayleigh-Ritz of the random block
  cholqr<double>(P, c, X, 1e-13, st);
  cholqr<double>(P, c, X, 1e-13, st);
  hx<double>(P, c, c.flags, OFF_X, NV_BLK, X, HX, nullptr, S, nullptr, 0, OUT_APPLY, st);
  CUDA_OK(cudaMemsetAsync(G3, 0, mat3, st));
  CUDA_OK(cudaMemsetAsync(A3, 0, mat3, st));
  launch_gram<double>(b, X, ox, NV_BLK, X, ox, NV_BLK, 4, nullptr, nullptr, G3, L3, st);
  launch_gram<double>(b, X, ox, NV_BLK, HX, ox, NV_BLK, 4, nullptr, nullptr, A3, L3, st);
  launch_rr_small(b, G3, A3, C3, th3, L3, NV_BLK, c.flags, st);
  launch_rotate<double, double>(b, X, ox, X, ox, NV_BLK, NV_BLK, 4, C3, L3, HX, HX, nullptr, nullptr, L3, st);
  bool have_p = false;
  for (int it = 0;; it++) {
    // residuals R = HX - X theta (into W) and the convergence test
    CUDA_OK(cudaMemsetAsync(r3, 0, size_t(M) * L3 * sizeof(double), st));
    launch_lobpcg_resid(b, X, HX, ox, th3, L3, W, r3, st);
    CUDA_OK(cudaMemsetAsync(c.active, 0, 4 * sizeof(int), st));
    launch_update_convergence(b, r3, L3, rs3, th3, c.bounds, prm->tol, 0.0, 0, c.prevres, c.stall, c.flags,
                              c.active, c.iters, st);
    CUDA_OK(cudaMemcpyAsync(ctx->h_active, c.active, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaStreamSynchronize(st));
    if (history) {
      double mx;
      std::memcpy(&mx, ctx->h_active + 2, sizeof(double));
      history[it] = mx;
    }
    if (*ctx->h_active == 0) break;
    if (it == prm->max_iter) {
      std::vector<int> hf(M), hc(M, 0);
      CUDA_OK(cudaMemcpy(hf.data(), c.flags, M * sizeof(int), cudaMemcpyDeviceToHost));
      for (int k = 0; k < M; k++) hc[k] = (hf[k] & EF_ACTIVE) ? 1 : 0;
      CUDA_OK(cudaMemcpy(c.hitcap, hc.data(), M * sizeof(int), cudaMemcpyHostToDevice));
      break;
    }
    // W = T R: Teter factor per band with E_v = <x_v, T x_v> dV (Eq. 3)
    launch_forward<double>(P.hx, ha, X, S, st);
    launch_zline<double>(P.hx, ha, S, MULT_KINETIC, st);
    launch_inverse_raw<double>(P.hx, ha, S, TX, st);
    CUDA_OK(cudaMemsetAsync(ek, 0, size_t(M) * L3 * sizeof(double), st));
    launch_vec_dots(b, X, TX, ox, L3, ek, st);
    HxArgs ht = ha;
    ht.mref = ek;
    ht.mref_ld = L3;
    launch_forward<double>(P.hx, ht, W, S, st);
    launch_zline<double>(P.hx, ht, S, MULT_TETER, st);
    launch_inverse_raw<double>(P.hx, ht, S, W, st);
    // unit rows of W (the span of the trial subspace is unchanged; S^T S stays well conditioned)
    CUDA_OK(cudaMemsetAsync(ek, 0, size_t(M) * L3 * sizeof(double), st));
    launch_vec_dots(b, W, W, ox, L3, ek, st);
    launch_scale_rows(b, W, nullptr, ox, ek, L3, st);
    hx<double>(P, c, c.flags, OFF_X, NV_BLK, W, HW, nullptr, S, nullptr, 0, OUT_APPLY, st);
    // projected problem over S = [X, W(, P)] (Eq. 5): Gram and H blocks, generalised Rayleigh-Ritz
    const int nb = have_p ? 3 : 2;
    const double* Sb[3] = {X, W, Pd};
    const double* Hb[3] = {HX, HW, HP};
    CUDA_OK(cudaMemsetAsync(G3, 0, mat3, st));
    CUDA_OK(cudaMemsetAsync(A3, 0, mat3, st));
    for (int i = 0; i < nb; i++)
      for (int j = 0; j < nb; j++) {
        const size_t o = size_t(i) * n * L3 + size_t(j) * n;
        launch_gram<double>(b, Sb[i], ox, NV_BLK, Sb[j], ox, NV_BLK, 4, nullptr, nullptr, G3 + o, L3, st);
        launch_gram<double>(b, Sb[i], ox, NV_BLK, Hb[j], ox, NV_BLK, 4, nullptr, nullptr, A3 + o, L3, st);
      }
    BatchArgs bp{have_p ? d3 : d2, c.flags, M};
    g_max_nblk = nb * n;
    launch_rr_small(bp, G3, A3, C3, th3, L3, NV_BLK, c.flags, st);
    g_max_nblk = n;
    // X = X C_X + P', P' = W C_W + P C_P (Eq. 4) and their H-images
    launch_lobpcg_update(b, ox, C3, L3, nb, X, W, Pd, HX, HW, HP, Xn, Pn, HXn, HPn, st);
    CUDA_OK(cudaMemsetAsync(ek, 0, size_t(M) * L3 * sizeof(double), st));
    launch_vec_dots(b, Pn, Pn, ox, L3, ek, st);
    launch_scale_rows(b, Pn, HPn, ox, ek, L3, st);   // unit rows of the next conjugate block
    std::swap(X, Xn);
    std::swap(HX, HXn);
    std::swap(Pd, Pn);
    std::swap(HP, HPn);
    have_p = true;
  }
  // Ritz values and residual norms in the result layout (ld P.L)
  CUDA_OK(cudaMemcpy2DAsync(c.theta, P.L * sizeof(double), th3, L3 * sizeof(double), P.L * sizeof(double), M,
                            cudaMemcpyDeviceToDevice, st));
  CUDA_OK(cudaMemcpy2DAsync(c.resid, P.L * sizeof(double), rs3, L3 * sizeof(double), P.L * sizeof(double), M,
                            cudaMemcpyDeviceToDevice, st));
  CUDA_OK(cudaGetLastError());
  *x_out = X;
  return DGDFT_OK;
}

}  // namespace dgdft

using namespace dgdft;

extern "C" {

int dgdft_alb_query_sizes(const dgdft_problem* prob, const dgdft_alb_params* params, int64_t out[6]) {
  if (!prob || !params || !out) return fail(nullptr, DGDFT_INVALID_ARG, "null argument");
  Plan P;
  std::string msg;
  int r = build_plan(prob, params, P, msg);
  if (r) return fail(nullptr, r, msg);
  out[0] = P.L;
  out[1] = P.tot[OFF_A];
  out[2] = P.tot[OFF_E];
  out[3] = int64_t(P.M) * P.L * P.L;
  out[4] = P.tot_grid;
  out[5] = int64_t(P.n_stencil) * P.M * P.L * P.L;
  return DGDFT_OK;
}

int dgdft_ctx_create(dgdft_ctx** out, int device) {
  if (!out) return fail(nullptr, DGDFT_INVALID_ARG, "null output pointer");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return fail(nullptr, DGDFT_CUDA_ERROR, std::string("no CUDA device ") + std::to_string(device) + ": " +
                                                cudaGetErrorString(e));
  }
  if (cudaSetDevice(device) != cudaSuccess) return fail(nullptr, DGDFT_CUDA_ERROR, "cudaSetDevice failed");
  dgdft_ctx* c = new dgdft_ctx();
  c->device = device;
  if (cudaMallocHost(&c->h_active, 4 * sizeof(int)) != cudaSuccess) {
    delete c;
    return fail(nullptr, DGDFT_CUDA_ERROR, "cudaMallocHost failed");
  }
  int r = init_twiddles(c);
  if (r) {
    cudaFreeHost(c->h_active);
    delete c;
    return r;
  }
  *out = c;
  return DGDFT_OK;
}

void dgdft_ctx_destroy(dgdft_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  for (auto& kv : c->bufs) cudaFree(kv.second.first);
  if (c->h_active) cudaFreeHost(c->h_active);
  delete c;
}

const char* dgdft_last_error(const dgdft_ctx* c) { return c ? c->err.c_str() : g_last_error.c_str(); }

int64_t dgdft_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int dgdft_stage_converged(double max_resid, double tol, double tol_mixed, int mixed, double b_up, double* prev_resid,
                          int* stall) {
  if (!prev_resid || !stall) return -DGDFT_INVALID_ARG;
  return stage_converged(max_resid, tol, tol_mixed, mixed, b_up, prev_resid, stall);
}

int dgdft_gram_fp32(dgdft_ctx* ctx, int n_blocks, const int* nx, const int* ny, const int* np, const double* dV,
                    const float* X, const int64_t* x_off, const float* Y, const int64_t* y_off, double* G, int ldg,
                    dgdft_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (!ctx || n_blocks < 0 || (n_blocks > 0 && (!nx || !ny || !np || !dV || !X || !x_off || !Y || !y_off || !G)))
    return fail(ctx, DGDFT_INVALID_ARG, "dgdft_gram_fp32: null argument or negative block count");
  if (n_blocks == 0) return DGDFT_OK;
  int max_rows = 0, max_np = 0;
  for (int k = 0; k < n_blocks; k++) {
    if (nx[k] < 0 || ny[k] < 0 || np[k] < 0 || nx[k] > 96 || ny[k] > 96 || nx[k] > ldg || ny[k] > ldg ||
        x_off[k] < 0 || y_off[k] < 0)
      return fail(ctx, DGDFT_INVALID_ARG, "dgdft_gram_fp32: block " + std::to_string(k) +
                                              ": rows outside 0..min(96, ldg) or a negative count or offset");
    max_rows = std::max(max_rows, std::max(nx[k], ny[k]));
    max_np = std::max(max_np, np[k]);
  }
  CUDA_OK(cudaSetDevice(ctx->device));
  // block k as an element descriptor: rows of X in n_blk, rows of Y in n_eig, points in N
  std::vector<ElemDesc> hd(n_blocks);
  std::vector<long long> ho(2 * n_blocks);
  for (int k = 0; k < n_blocks; k++) {
    hd[k] = ElemDesc{};
    hd[k].n_blk = nx[k];
    hd[k].n_eig = ny[k];
    hd[k].N = np[k];
    hd[k].dV = dV[k];
    ho[k] = x_off[k];
    ho[n_blocks + k] = y_off[k];
  }
  ElemDesc* dd = (ElemDesc*)ws(ctx, "gram_desc", n_blocks * sizeof(ElemDesc));
  long long* doff = (long long*)ws(ctx, "gram_off", 2 * n_blocks * sizeof(long long));
  if (!dd || !doff) return fail(ctx, DGDFT_OUT_OF_MEMORY, "dgdft_gram_fp32: workspace allocation failed");
  CUDA_OK(cudaMemcpyAsync(dd, hd.data(), n_blocks * sizeof(ElemDesc), cudaMemcpyHostToDevice, st));
  CUDA_OK(cudaMemcpyAsync(doff, ho.data(), 2 * n_blocks * sizeof(long long), cudaMemcpyHostToDevice, st));
  CUDA_OK(cudaMemsetAsync(G, 0, (size_t)n_blocks * ldg * ldg * sizeof(double), st));
  g_max_points = max_np;
  g_max_nblk = max_rows;
  g_max_nalb = 0;
  BatchArgs b{dd, nullptr, n_blocks};
  if (max_rows > 0 && max_np > 0 &&
      !launch_gram_tc(b, X, doff, NV_BLK, Y, doff + n_blocks, NV_EIG, 4, G, ldg, st, 1.0, max_rows))
    return fail(ctx, DGDFT_UNSUPPORTED, "dgdft_gram_fp32: block shape not handled");
  CUDA_OK(cudaGetLastError());
  CUDA_OK(cudaStreamSynchronize(st));
  if (take_tc_error()) return fail(ctx, DGDFT_CUDA_ERROR, "dgdft_gram_fp32: a tensor-core wait ran out");
  return DGDFT_OK;
}

int dgdft_rotate_fp32(dgdft_ctx* ctx, int n_blocks, const int* nin, const int* nout, const int* np, const float* X,
                      const int64_t* x_off, const double* W, int ldw, float* Z, const int64_t* z_off,
                      dgdft_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (!ctx || n_blocks < 0 || (n_blocks > 0 && (!nin || !nout || !np || !X || !x_off || !W || !Z || !z_off)))
    return fail(ctx, DGDFT_INVALID_ARG, "dgdft_rotate_fp32: null argument or negative block count");
  if (n_blocks == 0) return DGDFT_OK;
  int max_rows = 0, max_np = 0;
  for (int k = 0; k < n_blocks; k++) {
    if (nin[k] < 0 || nout[k] < 0 || np[k] < 0 || nin[k] > 96 || nout[k] > 96 || nin[k] > ldw || nout[k] > ldw ||
        x_off[k] < 0 || z_off[k] < 0)
      return fail(ctx, DGDFT_INVALID_ARG, "dgdft_rotate_fp32: block " + std::to_string(k) +
                                              ": vectors outside 0..min(96, ldw) or a negative count or offset");
    max_rows = std::max(max_rows, std::max(nin[k], nout[k]));
    max_np = std::max(max_np, np[k]);
  }
  CUDA_OK(cudaSetDevice(ctx->device));
  std::vector<ElemDesc> hd(n_blocks);
  std::vector<long long> ho(2 * n_blocks);
  for (int k = 0; k < n_blocks; k++) {
    hd[k] = ElemDesc{};
    hd[k].n_blk = nin[k];
    hd[k].n_eig = nout[k];
    hd[k].N = np[k];
    ho[k] = x_off[k];
    ho[n_blocks + k] = z_off[k];
  }
  ElemDesc* dd = (ElemDesc*)ws(ctx, "rot_desc", n_blocks * sizeof(ElemDesc));
  long long* doff = (long long*)ws(ctx, "rot_off", 2 * n_blocks * sizeof(long long));
  if (!dd || !doff) return fail(ctx, DGDFT_OUT_OF_MEMORY, "dgdft_rotate_fp32: workspace allocation failed");
  CUDA_OK(cudaMemcpyAsync(dd, hd.data(), n_blocks * sizeof(ElemDesc), cudaMemcpyHostToDevice, st));
  CUDA_OK(cudaMemcpyAsync(doff, ho.data(), 2 * n_blocks * sizeof(long long), cudaMemcpyHostToDevice, st));
  g_max_points = max_np;
  g_max_nblk = max_rows;
  g_max_nalb = 0;
  BatchArgs b{dd, nullptr, n_blocks};
  if (max_rows > 0 && max_np > 0 &&
      !launch_rotate_tc(b, X, doff, Z, doff + n_blocks, NV_BLK, NV_EIG, 4, W, ldw, nullptr, nullptr, nullptr, nullptr,
                        0, st, max_rows))
    return fail(ctx, DGDFT_UNSUPPORTED, "dgdft_rotate_fp32: block shape not handled");
  CUDA_OK(cudaGetLastError());
  CUDA_OK(cudaStreamSynchronize(st));
  if (take_tc_error()) return fail(ctx, DGDFT_CUDA_ERROR, "dgdft_rotate_fp32: a tensor-core wait ran out");
  return DGDFT_OK;
}

int dgdft_alb_generate(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* prm,
                       dgdft_alb_result* res, dgdft_stream stream) {
  if (!ctx || !prob || !prm || !res) return fail(ctx, DGDFT_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_OK(cudaSetDevice(ctx->device));
  Plan P;
  std::string msg;
  int r = build_plan(prob, prm, P, msg);
  if (r) return fail(ctx, r, msg);
  if (!res->eigval || !res->resid || !res->sing || !res->coef || !res->alb || !res->iters || !res->status)
    return fail(ctx, DGDFT_INVALID_ARG, "result arrays must be non-null (eigvec may be null)");
  const bool host = (prm->flags & DGDFT_HOST_BUFFERS) != 0;
  if (prm->solver != DGDFT_CHEFSI && prm->solver != DGDFT_LOBPCG)
    return fail(ctx, DGDFT_INVALID_ARG, "unknown solver");
  if (prm->solver == DGDFT_LOBPCG) {
    if (prm->precision != DGDFT_FP64) return fail(ctx, DGDFT_UNSUPPORTED, "LOBPCG runs in DGDFT_FP64");
    for (int k = 0; k < P.M; k++)
      if (P.desc[k].n_blk != P.desc[0].n_blk || P.desc[k].n_blk > 32)
        return fail(ctx, DGDFT_UNSUPPORTED, "LOBPCG needs the same block size <= 32 in every element");
  }
  const int degree = prm->cheb_degree;
  const int lsteps = prm->lanczos_steps > 0 ? prm->lanczos_steps : 10;
  if ((r = upload_plan(ctx, P, st))) return r;
  Common c;
  if ((r = get_common(ctx, P, degree, lsteps, c))) return r;
  const size_t M = P.M, L = P.L;
  // inputs
  const double* vx = prob->v_extra;
  if (host && vx) {
    double* d;
    WS(d, "vx_stage", P.tot_grid * sizeof(double));
    CUDA_OK(cudaMemcpyAsync(d, vx, P.tot_grid * sizeof(double), cudaMemcpyHostToDevice, st));
    vx = d;
  }
  const double* x0 = prm->x0;   // warm start [n_eig][N] per element (eigvec layout)
  if (host && x0) {
    double* d;
    WS(d, "x0_stage", P.tot[OFF_E] * sizeof(double));
    CUDA_OK(cudaMemcpyAsync(d, x0, P.tot[OFF_E] * sizeof(double), cudaMemcpyHostToDevice, st));
    x0 = d;
  }
  CUDA_OK(cudaMemsetAsync(c.flags, 0, M * sizeof(int), st));
  CUDA_OK(cudaMemsetAsync(c.iters, 0xFF, M * sizeof(int), st));   // -1: the start-up Rayleigh-Ritz is not a pass
  CUDA_OK(cudaMemsetAsync(c.stall, 0, M * sizeof(int), st));
  CUDA_OK(cudaMemsetAsync(c.hitcap, 0, M * sizeof(int), st));
  CUDA_OK(cudaMemsetAsync(c.bounds, 0, M * 3 * sizeof(double), st));
  {
    std::vector<double> big(M, 1e300);
    CUDA_OK(cudaMemcpyAsync(c.prevres, big.data(), M * sizeof(double), cudaMemcpyHostToDevice, st));
    CUDA_OK(cudaStreamSynchronize(st));
  }
  BatchArgs ball{P.d_desc, nullptr, P.M};
  launch_setup_v(ball, P.d_boxes, P.d_dtab, vx, P.r_cut, c.V64, c.V32, c.flags, st);
  launch_set_active(ball, c.flags, st);

  double* X64 = nullptr;
  Stage<double> s64;
  if (prm->precision == DGDFT_MIXED) {
    Stage<float> s32;
    const int u32[4] = {0, 1, 2, 3};
    if ((r = get_stage<float>(ctx, P, s32, 6, u32))) return r;
    launch_random_init<float>(ball, s32.B[0], P.d_off[OFF_X], prm->seed, st);
    if ((r = chefsi_stage<float>(ctx, P, c, s32, prm, degree, lsteps, true, st, res->history, x0))) return r;
    // final FP64 Rayleigh-Ritz sweep on the FP32 Ritz vectors: X64 in place, HX64 over B1/B2 of the FP32 stage.
    // The FP32 block is orthonormal only to FP32 accuracy; the Rayleigh-Ritz solve takes the Cholesky
    // factor of its FP64 Gram matrix (generalised problem), so no separate CholQR pass is needed.
    const int u64[4] = {4, 4, 4, 1};
    if ((r = get_stage<double>(ctx, P, s64, 6, u64))) return r;
    launch_set_active(ball, c.flags, st);
    BatchArgs b{P.d_desc, c.flags, P.M};
    const long long* ox = P.d_off[OFF_X];
    launch_convert<float, double>(b, s32.B[0], ox, s64.B[0], ox, NV_BLK, st);
    {
      // Rayleigh-Ritz in FP64: HX64 = H X64, G1 = X64^T X64 dV, G2 = X64^T HX64 dV, W (generalised)
      Stage<double>& s = s64;
      const size_t mat = size_t(P.M) * P.L * P.L * sizeof(double);
      hx<double>(P, c, c.flags, OFF_X, NV_BLK, s.B[0], s.HY, nullptr, s.S, nullptr, 0, OUT_APPLY, st);
      CUDA_OK(cudaMemsetAsync(c.G1, 0, mat, st));
      CUDA_OK(cudaMemsetAsync(c.G2, 0, mat, st));
      launch_gram<double>(b, s.B[0], ox, NV_BLK, s.B[0], ox, NV_BLK, 4, nullptr, nullptr, c.G1, P.L, st);
      launch_gram<double>(b, s.B[0], ox, NV_BLK, s.HY, ox, NV_BLK, 4, nullptr, nullptr, c.G2, P.L, st);
      launch_rr_small(b, c.G1, c.G2, c.W, c.theta, P.L, NV_BLK, c.flags, st);
      // residuals ||HX w - theta X w|| from FP32 copies (they sit at the FP32 floor): X32 is the FP32
      // block itself, HX32 goes to the free FP32 unit 3; then the FP64 rotation X64 W in place
      float* hx32 = s32.HY;
      launch_convert<double, float>(b, s.HY, ox, hx32, ox, NV_BLK, st);
      CUDA_OK(cudaMemsetAsync(c.resid2, 0, size_t(P.M) * P.L * sizeof(double), st));
      launch_rotate<float, float>(b, s32.B[0], ox, nullptr, ox, NV_BLK, NV_BLK, 4, c.W, P.L, hx32, nullptr, c.theta,
                                  c.resid2, P.L, st);
      launch_rotate<double, double>(b, s.B[0], ox, s.B[0], ox, NV_BLK, NV_BLK, 4, c.W, P.L, nullptr, nullptr, nullptr,
                                    nullptr, P.L, st);
    }
    launch_final_resid(b, c.resid2, P.L, c.resid, st);
    X64 = s64.B[0];
  } else if (prm->solver == DGDFT_LOBPCG) {
    const int u64[4] = {0, 2, 4, 6};
    if ((r = get_stage<double>(ctx, P, s64, 8, u64))) return r;
    launch_random_init<double>(ball, s64.B[0], P.d_off[OFF_X], prm->seed, st);
    if (x0) launch_convert<double, double>(ball, x0, P.d_off[OFF_E], s64.B[0], P.d_off[OFF_X], NV_EIG, st);
    if ((r = lobpcg_stage(ctx, P, c, prm, s64.B[0], st, res->history, &X64))) return r;
  } else {
    const int u64[4] = {0, 2, 4, 6};
    if ((r = get_stage<double>(ctx, P, s64, 8, u64))) return r;
    launch_random_init<double>(ball, s64.B[0], P.d_off[OFF_X], prm->seed, st);
    if ((r = chefsi_stage<double>(ctx, P, c, s64, prm, degree, lsteps, false, st, res->history, x0))) return r;
    X64 = s64.B[0];
  }
  CUDA_OK(cudaGetLastError());
  if (prm->precision != DGDFT_FP64) {
    CUDA_OK(cudaStreamSynchronize(st));
    if (take_tc_error()) return fail(ctx, DGDFT_CUDA_ERROR, "a bounded tensor-core wait of the FP32 Gram ran out");
  }

  // ---- outputs ----
  double *d_eigval = res->eigval, *d_resid = res->resid, *d_sing = res->sing, *d_coef = res->coef, *d_alb = res->alb;
  double* d_eigvec = res->eigvec;
  int *d_iters = res->iters, *d_status = res->status;
  if (host) {
    WS(d_eigval, "o_eigval", M * L * sizeof(double));
    WS(d_resid, "o_resid", M * L * sizeof(double));
    WS(d_sing, "o_sing", M * L * sizeof(double));
    WS(d_coef, "o_coef", M * L * L * sizeof(double));
    WS(d_alb, "o_alb", P.tot[OFF_A] * sizeof(double));
    WS(d_iters, "o_iters", M * sizeof(int));
    WS(d_status, "o_status", M * sizeof(int));
    d_eigvec = nullptr;
  }
  if (d_eigvec == nullptr) WS(d_eigvec, "eigvec_ws", P.tot[OFF_E] * sizeof(double));
  BatchArgs b{P.d_desc, nullptr, P.M};
  CUDA_OK(cudaMemcpyAsync(d_eigval, c.theta, M * L * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CUDA_OK(cudaMemcpyAsync(d_resid, c.resid, M * L * sizeof(double), cudaMemcpyDeviceToDevice, st));
  launch_convert<double, double>(b, X64, P.d_off[OFF_X], d_eigvec, P.d_off[OFF_E], NV_EIG, st);
  // ALB: restrict, Gram, eigen (descending) -> C, A = C^T Phi_E, display sign
  double* PhiE;
  WS(PhiE, "PhiE", P.tot[OFF_FE] * sizeof(double));
  launch_restrict(b, d_eigvec, P.d_off[OFF_E], PhiE, P.d_off[OFF_FE], NV_EIG, st);
  CUDA_OK(cudaMemsetAsync(c.G1, 0, M * L * L * sizeof(double), st));
  launch_gram<double>(b, PhiE, P.d_off[OFF_FE], NV_EIG, PhiE, P.d_off[OFF_FE], NV_EIG, 5, nullptr, nullptr, c.G1, P.L,
                      st);
  CUDA_OK(cudaMemsetAsync(d_sing, 0, M * L * sizeof(double), st));
  launch_svd_small(b, c.G1, d_coef, d_sing, P.L, P.L, st);
  launch_rotate<double, double>(b, PhiE, P.d_off[OFF_FE], d_alb, P.d_off[OFF_A], NV_EIG, NV_ALB, 5, d_coef, P.L,
                                nullptr, nullptr, nullptr, nullptr, P.L, st);
  launch_alb_sign(b, d_alb, P.d_off[OFF_A], d_coef, P.L, st);
  CUDA_OK(cudaMemcpyAsync(d_iters, c.iters, M * sizeof(int), cudaMemcpyDeviceToDevice, st));
  launch_elem_status(b, c.flags, c.resid, P.L, prm->tol, c.hitcap, d_status, st);
  CUDA_OK(cudaGetLastError());
  if (host) {
    CUDA_OK(cudaMemcpyAsync(res->eigval, d_eigval, M * L * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(res->resid, d_resid, M * L * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(res->sing, d_sing, M * L * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(res->coef, d_coef, M * L * L * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(res->alb, d_alb, P.tot[OFF_A] * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(res->iters, d_iters, M * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(res->status, d_status, M * sizeof(int), cudaMemcpyDeviceToHost, st));
  }
  CUDA_OK(cudaStreamSynchronize(st));
  std::vector<int> hs(M);
  if (!host) CUDA_OK(cudaMemcpy(hs.data(), d_status, M * sizeof(int), cudaMemcpyDeviceToHost));
  else std::memcpy(hs.data(), res->status, M * sizeof(int));
  int worst = DGDFT_OK;
  for (int k = 0; k < P.M; k++)
    if (hs[k] == DGDFT_BAD_INPUT) worst = DGDFT_BAD_INPUT;
    else if (hs[k] == DGDFT_CHOLESKY_FAIL && worst != DGDFT_BAD_INPUT) worst = DGDFT_CHOLESKY_FAIL;
    else if (hs[k] == DGDFT_NOT_CONVERGED && worst == DGDFT_OK) worst = DGDFT_NOT_CONVERGED;
  if (worst != DGDFT_OK) ctx->err = "see per-element status";
  return worst;
}

int dgdft_apply_hamiltonian(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* prm, const void* X,
                            void* Y, dgdft_stream stream) {
  if (!ctx || !prob || !prm || !X || !Y) return fail(ctx, DGDFT_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_OK(cudaSetDevice(ctx->device));
  Plan P;
  std::string msg;
  int r = build_plan(prob, prm, P, msg);
  if (r) return fail(ctx, r, msg);
  if ((r = upload_plan(ctx, P, st))) return r;
  Common c;
  if ((r = get_common(ctx, P, std::max(2, prm->cheb_degree), 10, c))) return r;
  CUDA_OK(cudaMemsetAsync(c.flags, 0, P.M * sizeof(int), st));
  BatchArgs ball{P.d_desc, nullptr, P.M};
  launch_setup_v(ball, P.d_boxes, P.d_dtab, prob->v_extra, P.r_cut, c.V64, c.V32, c.flags, st);
  cplx<double>* S;
  WS(S, "S_spec", size_t(P.tot[OFF_S]) * sizeof(cplx<double>));
  if (prm->precision == DGDFT_MIXED)
    hx<float>(P, c, nullptr, OFF_X, NV_BLK, (const float*)X, (float*)Y, nullptr, (cplx<float>*)S, nullptr, 0,
              OUT_APPLY, st);
  else
    hx<double>(P, c, nullptr, OFF_X, NV_BLK, (const double*)X, (double*)Y, nullptr, S, nullptr, 0, OUT_APPLY, st);
  CUDA_OK(cudaGetLastError());
  std::vector<int> hf(P.M);
  CUDA_OK(cudaMemcpyAsync(hf.data(), c.flags, P.M * sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_OK(cudaStreamSynchronize(st));
  for (int k = 0; k < P.M; k++)
    if (hf[k] & EF_BAD)
      return fail(ctx, DGDFT_BAD_INPUT, "element " + std::to_string(k) + ": v_extra is not finite on Q");
  return DGDFT_OK;
}

int dgdft_chebyshev_filter(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* prm,
                           const double* bounds, const void* X, void* Y, dgdft_stream stream) {
  if (!ctx || !prob || !prm || !X || !Y || !bounds) return fail(ctx, DGDFT_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_OK(cudaSetDevice(ctx->device));
  Plan P;
  std::string msg;
  int r = build_plan(prob, prm, P, msg);
  if (r) return fail(ctx, r, msg);
  if ((r = upload_plan(ctx, P, st))) return r;
  const int degree = prm->cheb_degree;
  Common c;
  if ((r = get_common(ctx, P, degree, 10, c))) return r;
  CUDA_OK(cudaMemsetAsync(c.flags, 0, P.M * sizeof(int), st));
  BatchArgs ball{P.d_desc, nullptr, P.M};
  launch_setup_v(ball, P.d_boxes, P.d_dtab, prob->v_extra, P.r_cut, c.V64, c.V32, c.flags, st);
  CUDA_OK(cudaMemcpyAsync(c.bounds, bounds, P.M * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
  launch_cheb_coeffs(ball, c.bounds, c.cheb, degree, st);
  auto run = [&](auto tag) -> int {
    using T = decltype(tag);
    Stage<T> s;
    const int f = sizeof(T) / 4;
    const int uu[4] = {0, f, 2 * f, 3 * f};
    int rr = get_stage<T>(ctx, P, s, 4 * f, uu);
    if (rr) return rr;
    const long long* ox = P.d_off[OFF_X];
    T* x = (T*)const_cast<void*>(X);
    // HX into the stage's HY, step 1 into B1, then the recurrence; result copied to Y
    hx<T>(P, c, nullptr, OFF_X, NV_BLK, x, s.HY, nullptr, s.S, nullptr, 0, OUT_APPLY, st);
    launch_cheb_first<T>(ball, x, s.HY, s.B[1], ox, c.cheb, 3 * degree, st);
    T* prev = x;
    T* cur = s.B[1];
    T* spare = s.B[2];
    for (int step = 1; step < degree; step++) {
      hx<T>(P, c, nullptr, OFF_X, NV_BLK, cur, spare, prev, s.S, c.cheb + 3 * step, 3 * degree, OUT_CHEB, st);
      T* t = prev;
      prev = cur;
      cur = spare;
      spare = (t == x) ? s.B[0] : t;
    }
    cudaMemcpyAsync(Y, cur, P.tot[OFF_X] * sizeof(T), cudaMemcpyDeviceToDevice, st);
    return DGDFT_OK;
  };
  r = prm->precision == DGDFT_MIXED ? run(float()) : run(double());
  if (r) return r;
  CUDA_OK(cudaGetLastError());
  CUDA_OK(cudaStreamSynchronize(st));
  return DGDFT_OK;
}

}  // extern "C"

namespace dgdft {

// Element-local DG ingredients (Eq. DGHamiltonian): KV = kinetic + V_eff part of the diagonal block
// [M][L][L], face traces TR (packed per element at desc.troff) and projector overlaps on E, PE (packed
// at desc.peoff).  Every pointer is a device pointer.
static int dg_ingredients_dev(dgdft_ctx* ctx, Plan& P, const Common& c, const double* eigvec, const double* coef,
                              const double* vx, double* KV, double* TR, double* PE, cudaStream_t st) {
  const size_t M = P.M, L = P.L;
  BatchArgs b{P.d_desc, nullptr, P.M};
  CUDA_OK(cudaMemsetAsync(c.flags, 0, M * sizeof(int), st));
  launch_setup_v(b, P.d_boxes, P.d_dtab, vx, P.r_cut, c.V64, c.V32, c.flags, st);
  // psi^Q = C^T Phi^Q (trig interpolant of the ALBs on Q), its restriction A to E
  double *Psi, *D, *PsiE, *VE;
  cplx<double>* S;
  {
    char* ar = arena(ctx, P, 4);
    if (!ar) return fail(ctx, DGDFT_OUT_OF_MEMORY, "out of device memory: block arena");
    Psi = (double*)ar;
    D = (double*)(ar + 2 * size_t(P.tot[OFF_X]) * 4);
  }
  WS(PsiE, "PhiE", P.tot[OFF_FE] * sizeof(double));
  WS(VE, "dg_ve", P.tot[OFF_VE] * sizeof(double));
  WS(S, "S_spec", size_t(P.tot[OFF_S]) * sizeof(cplx<double>));
  const long long* oe = P.d_off[OFF_E];
  const long long* ofe = P.d_off[OFF_FE];
  launch_rotate<double, double>(b, eigvec, oe, Psi, oe, NV_EIG, NV_ALB, 4, coef, P.L, nullptr, nullptr, nullptr,
                                nullptr, P.L, st);
  // kinetic: 1/2 sum_axes (d psi)_E^T (d psi)_E dV with spectral derivatives (Nyquist dropped)
  CUDA_OK(cudaMemsetAsync(KV, 0, M * L * L * sizeof(double), st));
  set_group_nvec(P, NV_ALB);
  HxArgs ha = hx_args(P, nullptr, OFF_E, NV_ALB);
  // one forward pass along x and y for the three axes: d/dx and d/dy need no z transform (their multiplier
  // does not depend on k_z) and are applied as the inverse pass reads the spectrum; d/dz last, in place
  launch_forward<double>(P.hx, ha, Psi, S, st);
  for (int axis = 0; axis < 3; axis++) {
    if (axis == 2) launch_zline<double>(P.hx, ha, S, MULT_DZ, st);
    launch_inverse_raw<double>(P.hx, ha, S, D, st, axis < 2 ? axis : -1);
    launch_restrict(b, D, oe, PsiE, ofe, NV_ALB, st);
    launch_gram<double>(b, PsiE, ofe, NV_ALB, PsiE, ofe, NV_ALB, 5, nullptr, nullptr, KV, P.L, st, 0.5);
  }
  // V_eff term: A diag(V_E) A^T dV with A = psi restricted to E
  launch_restrict(b, c.V64, P.d_off[OFF_V], VE, P.d_off[OFF_VE], NV_ONE, st);
  launch_restrict(b, Psi, oe, PsiE, ofe, NV_ALB, st);
  launch_gram<double>(b, PsiE, ofe, NV_ALB, PsiE, ofe, NV_ALB, 5, VE, P.d_off[OFF_VE], KV, P.L, st);
  // projector overlaps on E and face traces
  if (P.tot_pe > 0) CUDA_OK(cudaMemsetAsync(PE, 0, P.tot_pe * sizeof(double), st));
  launch_proj_overlap(b, P.d_boxes, P.d_dtab, PsiE, ofe, P.r_cut, P.n_proj_per_atom, PE, P.max_pe, st);
  if (P.tot_tr > 0) {
    CUDA_OK(cudaMemsetAsync(TR, 0, P.tot_tr * sizeof(double), st));
    launch_face_traces(b, Psi, oe, TR, st);
  }
  CUDA_OK(cudaGetLastError());
  return DGDFT_OK;
}

// Blocks from the ingredients (device pointers): the stencil of every element of the plan.
static int dg_blocks_dev(dgdft_ctx* ctx, Plan& P, const dgdft_problem* prob, const double* KV, const double* TR,
                         const double* PE, double alpha, double* out, cudaStream_t st) {
  const size_t M = P.M;
  int* d_nb;
  WS(d_nb, "dg_nb", std::max<size_t>(1, M * P.n_stencil) * sizeof(int));
  {
    std::vector<int> nb(M * P.n_stencil);
    for (size_t k = 0; k < M; k++)
      for (int s = 0; s < P.n_stencil; s++)
        nb[k * P.n_stencil + s] = P.n_stencil > 1 ? prob->neighbors[k * P.n_stencil + s] : int(k);
    CUDA_OK(cudaMemcpyAsync(d_nb, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  BatchArgs b{P.d_desc, nullptr, P.M};
  launch_dg_blocks(b, d_nb, P.n_stencil, TR, PE, P.d_boxes, P.n_proj_per_atom, KV, P.L, alpha, out, st);
  CUDA_OK(cudaGetLastError());
  return DGDFT_OK;
}

static int dg_eigvec(dgdft_ctx* ctx, const Plan& P, const dgdft_alb_result* res, bool host, const double** out) {
  const double* eigvec = (host || res->eigvec == nullptr) ? nullptr : res->eigvec;
  if (!eigvec) {
    auto it = ctx->bufs.find("eigvec_ws");
    if (it == ctx->bufs.end() || it->second.second < size_t(P.tot[OFF_E]) * sizeof(double))
      return fail(ctx, DGDFT_INVALID_ARG, "no eigenvectors: pass result->eigvec or call dgdft_alb_generate first");
    eigvec = (const double*)it->second.first;
  }
  *out = eigvec;
  return DGDFT_OK;
}

// Stages a host array into a named workspace buffer (host == true) or returns the device pointer as is.
static int stage_in(dgdft_ctx* ctx, bool host, const char* name, const double* src, size_t n, const double** out,
                    cudaStream_t st) {
  if (!host || src == nullptr) {
    *out = src;
    return DGDFT_OK;
  }
  double* d;
  WS(d, name, std::max<size_t>(1, n) * sizeof(double));
  if (n) CUDA_OK(cudaMemcpyAsync(d, src, n * sizeof(double), cudaMemcpyHostToDevice, st));
  *out = d;
  return DGDFT_OK;
}

}  // namespace dgdft

extern "C" {

int dgdft_dg_query_layout(const dgdft_problem* prob, const dgdft_alb_params* params, int64_t* tr_off,
                          int64_t* pe_off) {
  if (!prob || !params || !tr_off || !pe_off) return fail(nullptr, DGDFT_INVALID_ARG, "null argument");
  Plan P;
  std::string msg;
  int r = build_plan(prob, params, P, msg);
  if (r) return fail(nullptr, r, msg);
  for (int k = 0; k < P.M; k++) {
    tr_off[k] = P.desc[k].troff;
    pe_off[k] = P.desc[k].peoff;
  }
  tr_off[P.M] = P.tot_tr;
  pe_off[P.M] = P.tot_pe;
  return DGDFT_OK;
}

int dgdft_dg_ingredients(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* prm,
                         const dgdft_alb_result* res, double* kv, double* traces, double* proj, dgdft_stream stream) {
  if (!ctx || !prob || !prm || !res || !res->coef || !kv || !traces || !proj)
    return fail(ctx, DGDFT_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_OK(cudaSetDevice(ctx->device));
  Plan P;
  std::string msg;
  int r = build_plan(prob, prm, P, msg);
  if (r) return fail(ctx, r, msg);
  const bool host = (prm->flags & DGDFT_HOST_BUFFERS) != 0;
  if ((r = upload_plan(ctx, P, st))) return r;
  Common c;
  if ((r = get_common(ctx, P, std::max(2, prm->cheb_degree), 10, c))) return r;
  const size_t M = P.M, L = P.L;
  const double *eigvec, *coef, *vx;
  if ((r = dg_eigvec(ctx, P, res, host, &eigvec))) return r;
  if ((r = stage_in(ctx, host, "dg_coef", res->coef, M * L * L, &coef, st))) return r;
  if ((r = stage_in(ctx, host, "vx_stage", prob->v_extra, P.tot_grid, &vx, st))) return r;
  double *KV = kv, *TR = traces, *PE = proj;
  if (host) {
    WS(KV, "dg_kv", M * L * L * sizeof(double));
    WS(TR, "dg_tr", std::max<long long>(1, P.tot_tr) * sizeof(double));
    WS(PE, "dg_pe", std::max<long long>(1, P.tot_pe) * sizeof(double));
  }
  if ((r = dg_ingredients_dev(ctx, P, c, eigvec, coef, vx, KV, TR, PE, st))) return r;
  if (host) {
    CUDA_OK(cudaMemcpyAsync(kv, KV, M * L * L * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (P.tot_tr) CUDA_OK(cudaMemcpyAsync(traces, TR, P.tot_tr * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (P.tot_pe) CUDA_OK(cudaMemcpyAsync(proj, PE, P.tot_pe * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CUDA_OK(cudaStreamSynchronize(st));
  return DGDFT_OK;
}

int dgdft_dg_blocks(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* prm, const double* kv,
                    const double* traces, const double* proj, double alpha, double* blocks, dgdft_stream stream) {
  if (!ctx || !prob || !prm || !kv || !traces || !proj || !blocks) return fail(ctx, DGDFT_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_OK(cudaSetDevice(ctx->device));
  Plan P;
  std::string msg;
  int r = build_plan(prob, prm, P, msg);
  if (r) return fail(ctx, r, msg);
  const bool host = (prm->flags & DGDFT_HOST_BUFFERS) != 0;
  if ((r = upload_plan(ctx, P, st))) return r;
  const size_t M = P.M, L = P.L;
  const double *KV, *TR, *PE;
  if ((r = stage_in(ctx, host, "dg_kv", kv, M * L * L, &KV, st))) return r;
  if ((r = stage_in(ctx, host, "dg_tr", traces, P.tot_tr, &TR, st))) return r;
  if ((r = stage_in(ctx, host, "dg_pe", proj, P.tot_pe, &PE, st))) return r;
  double* out = blocks;
  if (host) WS(out, "dg_blocks", size_t(P.n_stencil) * M * L * L * sizeof(double));
  if ((r = dg_blocks_dev(ctx, P, prob, KV, TR, PE, alpha, out, st))) return r;
  if (host)
    CUDA_OK(cudaMemcpyAsync(blocks, out, size_t(P.n_stencil) * M * L * L * sizeof(double), cudaMemcpyDeviceToHost,
                            st));
  CUDA_OK(cudaStreamSynchronize(st));
  return DGDFT_OK;
}

int dgdft_dg_assemble(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* prm,
                      const dgdft_alb_result* res, double alpha, double* blocks, dgdft_stream stream) {
  if (!ctx || !prob || !prm || !res || !blocks || !res->coef) return fail(ctx, DGDFT_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_OK(cudaSetDevice(ctx->device));
  Plan P;
  std::string msg;
  int r = build_plan(prob, prm, P, msg);
  if (r) return fail(ctx, r, msg);
  const bool host = (prm->flags & DGDFT_HOST_BUFFERS) != 0;
  if ((r = upload_plan(ctx, P, st))) return r;
  Common c;
  if ((r = get_common(ctx, P, std::max(2, prm->cheb_degree), 10, c))) return r;
  const size_t M = P.M, L = P.L;
  const double *eigvec, *coef, *vx;
  if ((r = dg_eigvec(ctx, P, res, host, &eigvec))) return r;
  if ((r = stage_in(ctx, host, "dg_coef", res->coef, M * L * L, &coef, st))) return r;
  if ((r = stage_in(ctx, host, "vx_stage", prob->v_extra, P.tot_grid, &vx, st))) return r;
  double* out = blocks;
  if (host) WS(out, "dg_blocks", size_t(P.n_stencil) * M * L * L * sizeof(double));
  double *PE, *TR;
  WS(PE, "dg_pe", std::max<long long>(1, P.tot_pe) * sizeof(double));
  WS(TR, "dg_tr", std::max<long long>(1, P.tot_tr) * sizeof(double));
  if ((r = dg_ingredients_dev(ctx, P, c, eigvec, coef, vx, c.G1, TR, PE, st))) return r;
  if ((r = dg_blocks_dev(ctx, P, prob, c.G1, TR, PE, alpha, out, st))) return r;
  if (host)
    CUDA_OK(cudaMemcpyAsync(blocks, out, size_t(P.n_stencil) * M * L * L * sizeof(double), cudaMemcpyDeviceToHost,
                            st));
  CUDA_OK(cudaStreamSynchronize(st));
  return DGDFT_OK;
}

int dgdft_alb_grad(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* prm,
                   const dgdft_alb_result* res, double kT, const double* n_electrons, double* energy, double* grad_v,
                   double* grad_R, dgdft_stream stream) {
  if (!ctx || !prob || !prm || !res || !n_electrons || !energy || !grad_v || !grad_R || !res->eigval)
    return fail(ctx, DGDFT_INVALID_ARG, "null argument");
  if (!(kT > 0)) return fail(ctx, DGDFT_INVALID_ARG, "kT must be positive");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_OK(cudaSetDevice(ctx->device));
  Plan P;
  std::string msg;
  int r = build_plan(prob, prm, P, msg);
  if (r) return fail(ctx, r, msg);
  const bool host = (prm->flags & DGDFT_HOST_BUFFERS) != 0;
  if ((r = upload_plan(ctx, P, st))) return r;
  Common c;
  if ((r = get_common(ctx, P, std::max(2, prm->cheb_degree), 10, c))) return r;
  const size_t M = P.M, L = P.L;
  const double* eigvec = (host || res->eigvec == nullptr) ? nullptr : res->eigvec;
  if (!eigvec) {
    auto it = ctx->bufs.find("eigvec_ws");
    if (it == ctx->bufs.end() || it->second.second < size_t(P.tot[OFF_E]) * sizeof(double))
      return fail(ctx, DGDFT_INVALID_ARG, "no eigenvectors: pass result->eigvec or call dgdft_alb_generate first");
    eigvec = (const double*)it->second.first;
  }
  const double* theta = res->eigval;
  double *d_E = energy, *d_gv = grad_v, *d_gR = grad_R;
  if (host) {
    double* t;
    WS(t, "gr_theta", M * L * sizeof(double));
    CUDA_OK(cudaMemcpyAsync(t, theta, M * L * sizeof(double), cudaMemcpyHostToDevice, st));
    theta = t;
    WS(d_E, "gr_E", M * sizeof(double));
    WS(d_gv, "gr_gv", P.tot_grid * sizeof(double));
    WS(d_gR, "gr_gR", std::max(1, prob->n_atoms) * 3 * sizeof(double));
  }
  double *nel, *w, *rho;
  WS(nel, "gr_nel", M * sizeof(double));
  WS(w, "gr_w", M * L * sizeof(double));
  WS(rho, "gr_rho", P.tot[OFF_V] * sizeof(double));
  CUDA_OK(cudaMemcpyAsync(nel, n_electrons, M * sizeof(double), cudaMemcpyHostToDevice, st));
  CUDA_OK(cudaMemsetAsync(c.flags, 0, M * sizeof(int), st));
  CUDA_OK(cudaMemsetAsync(d_gv, 0, P.tot_grid * sizeof(double), st));
  CUDA_OK(cudaMemsetAsync(d_gR, 0, std::max(1, prob->n_atoms) * 3 * sizeof(double), st));
  BatchArgs b{P.d_desc, nullptr, P.M};
  launch_fermi_weights(b, theta, P.L, nel, kT, w, d_E, c.flags, st);
  launch_density_scatter(b, eigvec, P.d_off[OFF_E], w, P.L, rho, P.d_off[OFF_V], d_gv, st);
  launch_atom_forces(b, P.d_boxes, P.d_dtab, eigvec, P.d_off[OFF_E], w, P.L, rho, P.d_off[OFF_V], P.r_cut,
                     P.n_proj_per_atom, d_gR, P.max_pa, st);
  CUDA_OK(cudaGetLastError());
  if (host) {
    CUDA_OK(cudaMemcpyAsync(energy, d_E, M * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(grad_v, d_gv, P.tot_grid * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(grad_R, d_gR, prob->n_atoms * 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  std::vector<int> hf(M);
  CUDA_OK(cudaMemcpyAsync(hf.data(), c.flags, M * sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_OK(cudaStreamSynchronize(st));
  for (size_t k = 0; k < M; k++)
    if (hf[k] & EF_BAD)
      return fail(ctx, DGDFT_BAD_INPUT, "element " + std::to_string(k) +
                                            ": the highest eigenpair is occupied (f >= 1e-12); enlarge n_eig");
  return DGDFT_OK;
}

}  // extern "C"
