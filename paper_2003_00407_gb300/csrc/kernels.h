// Launch interfaces of the CUDA kernels (host side).
#pragma once
#include <vector>
#include "internal.h"

namespace dgdft {

// line transforms n = 1..kMaxLine; twiddle table entry n(n-1)/2 + m = exp(-2 pi i m / n)
constexpr int kMaxLine = 64;
constexpr int kTwiddleCount = kMaxLine * (kMaxLine + 1) / 2;
__host__ __device__ constexpr int twiddle_offset(int n) { return n * (n - 1) / 2; }
int upload_twiddles(const double2* t64, const float2* t32);
int upload_fused_twiddles(const float2* t32);
constexpr int kFusedAtomLimit = 96;

// Kernel launches issued by this library since it was loaded (reported by dgdft_kernel_launches).
extern long long g_launches;
inline void count_launch() { __atomic_add_fetch(&g_launches, 1, __ATOMIC_RELAXED); }

// spectral multipliers of the multi-pass transforms: kinetic 1/2|G|^2, plain 1/N, d/dx, d/dy, d/dz, and the
// Teter preconditioner K(1/2|G|^2 / E_v) with E_v = HxArgs::mref[k * mref_ld + v]
enum MultMode { MULT_KINETIC = 0, MULT_SCALE = 1, MULT_DX = 2, MULT_DY = 3, MULT_DZ = 4, MULT_TETER = 5 };
enum OutMode { OUT_APPLY = 0, OUT_CHEB = 1, OUT_RAW = 2 };
enum NvecMode { NV_BLK = 0, NV_EIG = 1, NV_ALB = 2, NV_ONE = 3 };

struct HxArgs {
  const ElemDesc* desc;
  const int* elems;
  const int* flags;
  const AtomBox* boxes;
  const double* dtab;
  const long long* xo;   // per-element offset of the [nvec][N] blocks
  const long long* so;   // per-element offset of the spectra
  int nvec_mode;
  int n_proj_per_atom;
  double r_cut;
  const FusedAtomRec* fatoms;  // atom records of the fused kernel
  ProjList plist;              // their compact projector-point lists
  const double* mref;          // MULT_TETER: per (element, vector) reference kinetic energy
  int mref_ld;
};

struct ShapeGroup {
  int qn[3];
  int n_elems;
  int max_nvec;          // set by the launcher for the current mode
  int max_nblk, max_neig, max_nalb;
  int zchunk;
  bool fused_ok;         // every element's atom boxes fit the fused kernel's tables
  int* d_elems;          // device list of element ids
  std::vector<int> elems;
};

struct HxPlan {
  std::vector<ShapeGroup> groups;
};

int fused_shape_supported(const int qn[3]);
int set_fused_smem_limits();   // per device; returns the cudaError_t
// compact projector-point lists of the fused atom records (k_fused.cu), once per plan
void launch_build_proj_lists(const FusedAtomRec* fat, const double* dtab, int n, double r_cut, ProjList pl,
                             cudaStream_t st);
// fused FP32 Chebyshev step (k_fused.cu): returns 1 when it handled the group
int launch_fused_group(const ShapeGroup& g, const HxArgs& h, const float* X, float* Y, const float* Yprev,
                       const float* V, const double* cheb, int cheb_stride, int out_mode, cudaStream_t st);

int plane_smem_bytes(int qx, int qy, int elem_bytes);
// Raise a kernel's dynamic shared-memory limit to the device opt-in maximum
// minus the kernel's static shared memory.  Returns the cudaError_t.
template <typename F> int allow_max_smem(F* func) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return int(e);
  return int(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin - int(fa.sharedSizeBytes)));
}
int zline_smem_bytes(int qz, int chunk, int elem_bytes);
int set_hx_smem_limits();
int set_linalg_smem_limits();

template <typename T>
void launch_hx(const HxPlan& pl, const HxArgs& args, const T* X, T* Y, const T* Yprev, const T* V, cplx<T>* S,
               double* P, const double* cheb, int cheb_stride, int out_mode, int mult_mode, cudaStream_t st);
template <typename T>
void launch_forward(const HxPlan& pl, const HxArgs& args, const T* X, cplx<T>* S, cudaStream_t st);
template <typename T>
void launch_zline(const HxPlan& pl, const HxArgs& args, cplx<T>* S, int mult_mode, cudaStream_t st);
template <typename T>
// inverse transform of a spectrum (unnormalised); deriv = 0 / 1 applies d/dx / d/dy to a spectrum that
// was transformed along x and y only (the forward plane pass), deriv = -1 nothing
void launch_inverse_raw(const HxPlan& pl, const HxArgs& args, const cplx<T>* S, T* Y, cudaStream_t st, int deriv = -1);

// ---- batched per-element dense kernels (k_linalg.cu) ----
struct BatchArgs {
  const ElemDesc* desc;
  const int* flags;      // may be null
  int M;
};
// Gram matrices of FP32 blocks on the tensor cores (3xTF32, k_gram_tc.cu); 0 when the shape is not handled
int launch_gram_tc(const BatchArgs& b, const float* A, const long long* ao, int na_mode, const float* B,
                   const long long* bo, int nb_mode, int npts_mode, double* G, int ldg, cudaStream_t st,
                   double scale, int max_rows);
// subspace rotation of FP32 blocks on the tensor cores (3xTF32, k_gram_tc.cu); 0 when the shape is not handled
int launch_rotate_tc(const BatchArgs& b, const float* X, const long long* xo, float* Z, const long long* zo,
                     int nin_mode, int nout_mode, int npts_mode, const double* W, int ldw, const float* X2, float* Z2,
                     const double* theta, double* resid2, int ldr, cudaStream_t st, int max_rows);
int take_tc_error();   // 1 when a bounded tensor-core wait ran out since the last call (clears the flag)

// G_k[i][j] += dV * sum_p A_k[i][p] w(p) B_k[j][p]   (i < na, j < nb; ld = ldg)
template <typename TI>
void launch_gram(const BatchArgs& b, const TI* A, const long long* ao, int na_mode, const TI* B, const long long* bo,
                 int nb_mode, int npts_mode, const double* weight, const long long* wo, double* G, int ldg,
                 cudaStream_t st, double scale = 1.0);
// Z_k[j][p] = sum_i W_k[i][j] X_k[i][p] (in place allowed), optional second block and residuals
template <typename TX, typename TZ>
void launch_rotate(const BatchArgs& b, const TX* X, const long long* xo, TZ* Z, const long long* zo, int nin_mode,
                   int nout_mode, int npts_mode, const double* W, int ldw, const TX* X2, TZ* Z2, const double* theta,
                   double* resid2, int ldr, cudaStream_t st);
// small dense ops, one CTA per element
void launch_chol_inv(const BatchArgs& b, const double* S, double* Uinv, int ld, int n_mode, double rel_shift,
                     int* flags, cudaStream_t st);
void launch_rr_small(const BatchArgs& b, const double* S2, const double* G, double* W, double* theta, int ld,
                     int n_mode, int* flags, cudaStream_t st);
void launch_svd_small(const BatchArgs& b, const double* G, double* C, double* sing, int ld, int ldc,
                      cudaStream_t st);
// elementwise helpers
template <typename T>
void launch_random_init(const BatchArgs& b, T* X, const long long* xo, unsigned long long seed, cudaStream_t st);
template <typename T>
void launch_cheb_first(const BatchArgs& b, const T* X, const T* HX, T* Y, const long long* xo, const double* cheb,
                       int cheb_stride, cudaStream_t st);
// per-element coefficients of a filter of `degree` steps; with pdeg, element k stops after pdeg[k] steps
void launch_cheb_coeffs(const BatchArgs& b, const double* bounds, double* cheb, int degree, cudaStream_t st,
                        const int* pdeg = nullptr);
template <typename TS, typename TD>
void launch_convert(const BatchArgs& b, const TS* X, const long long* xo, TD* Y, const long long* yo, int nvec_mode,
                    cudaStream_t st);
void launch_setup_v(const BatchArgs& b, const AtomBox* boxes, const double* dtab, const double* v_extra, double r_cut,
                    double* V64, float* V32, int* flags, cudaStream_t st);
void launch_restrict(const BatchArgs& b, const double* X, const long long* xo, double* XE, const long long* eo,
                     int nvec_mode, cudaStream_t st);
void launch_alb_sign(const BatchArgs& b, double* A, const long long* ao, double* C, int ldc, cudaStream_t st);
// filter degree of the next pass per element (pdeg) and for the batch (out = max over active elements)
void launch_pass_degree(const BatchArgs& b, const double* bounds, int max_degree, double range_log, int* pdeg,
                        int* out, cudaStream_t st);
void launch_update_convergence(const BatchArgs& b, const double* resid2, int ldr, double* resid, const double* theta,
                               double* bounds, double tol, double tol_mixed, int mixed, double* prev_res,
                               int* stall, int* flags, int* active_count, int* iters, cudaStream_t st);
// Lanczos upper bound
template <typename T>
void launch_dot(const BatchArgs& b, const T* X, const T* Y, const long long* o, double* out, int ostride,
                cudaStream_t st);
template <typename T>
void launch_lanczos_update(const BatchArgs& b, T* v, T* f, T* vold, const long long* o, const double* alpha,
                           const double* beta_prev, int stride, int first, cudaStream_t st);
void launch_store_sqrt(const BatchArgs& b, const double* src, double* dst, int stride, cudaStream_t st);
void launch_final_resid(const BatchArgs& b, const double* resid2, int ldr, double* resid, cudaStream_t st);
void launch_set_active(const BatchArgs& b, int* flags, cudaStream_t st);
void launch_elem_status(const BatchArgs& b, const int* flags, const double* resid, int ldr, double tol,
                        const int* hit_cap, int* status, cudaStream_t st);
template <typename T>
void launch_scale_vec_old(const BatchArgs& b, T* v, const T* f, T* vold, const long long* o, const double* nrm2,
                          cudaStream_t st);
// per-call sizes of the current plan (set by the entry point on the calling host thread)
extern thread_local int g_max_points, g_max_nblk, g_max_nalb;
void launch_lanczos_bound(const BatchArgs& b, const double* alphas, const double* betas, int steps,
                          const double* fnorm2, double* bounds, double* lanczos_min, cudaStream_t st);
void launch_first_a0(const BatchArgs& b, const double* lanczos_min, double* bounds, cudaStream_t st);

// ---- LOBPCG local solver (k_lobpcg.cu) ----
void launch_lobpcg_resid(const BatchArgs& b, const double* X, const double* HX, const long long* xo,
                         const double* theta, int ld, double* W, double* resid2, cudaStream_t st);
void launch_vec_dots(const BatchArgs& b, const double* X, const double* Y, const long long* xo, int ld, double* out,
                     cudaStream_t st);
void launch_scale_rows(const BatchArgs& b, double* X, double* Y, const long long* xo, const double* nrm2, int ld,
                       cudaStream_t st);
void launch_lobpcg_update(const BatchArgs& b, const long long* xo, const double* C, int ld, int nb, const double* X,
                          const double* W, const double* P, const double* HX, const double* HW, const double* HP,
                          double* Xn, double* Pn, double* HXn, double* HPn, cudaStream_t st);

// ---- DG assembly (k_dg.cu) ----
void launch_proj_overlap(const BatchArgs& b, const AtomBox* boxes, const double* dtab, const double* A,
                         const long long* ao, double r_cut, int n_proj_per_atom, double* PE, int max_boxes,
                         cudaStream_t st);
void launch_face_traces(const BatchArgs& b, const double* Psi, const long long* po, double* TR, cudaStream_t st);
void launch_dg_blocks(const BatchArgs& b, const int* neighbors, int n_stencil, const double* TR, const double* PE,
                      const AtomBox* boxes, int n_proj_per_atom, const double* KV, int ld, double alpha,
                      double* blocks, cudaStream_t st);
// ---- gradient (k_grad.cu) ----
void launch_fermi_weights(const BatchArgs& b, const double* theta, int ld, const double* n_el, double kT,
                          double* w, double* energy, int* flags, cudaStream_t st);
void launch_density_scatter(const BatchArgs& b, const double* Phi, const long long* po, const double* w, int ld,
                            double* rho, const long long* ro, double* grad_v, cudaStream_t st);
void launch_atom_forces(const BatchArgs& b, const AtomBox* boxes, const double* dtab, const double* Phi,
                        const long long* po, const double* w, int ld, const double* rho, const long long* ro,
                        double r_cut, int n_proj_per_atom, double* grad_R, int max_boxes, cudaStream_t st);

}  // namespace dgdft
