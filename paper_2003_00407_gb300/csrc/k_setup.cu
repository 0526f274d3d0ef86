// Set-up and elementwise kernels: V_eff on Q (Eq. LocalKS), the counter-based
// random start, Chebyshev filter coefficients (Alg. CheFSI step 2), the
// Lanczos upper bound (step 1), convergence bookkeeping, restriction to E and
// the display sign of the ALBs.
#include "kernels.h"
#include "convergence.h"

namespace dgdft {

__device__ __forceinline__ int nvec_of(const ElemDesc& d, int mode) {
  return mode == 0 ? d.n_blk : (mode == 1 ? d.n_eig : (mode == 2 ? d.n_alb : 1));
}

// ---- V_eff on Q: gathered v_extra plus the Gaussian wells of the atom boxes ----
__global__ void k_setup_v(BatchArgs b, const AtomBox* boxes, const double* dtab, const double* v_extra, double r_cut,
                          double* V64, float* V32, int* flags) {
  const int k = blockIdx.y;
  const ElemDesc& d = b.desc[k];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.N) return;
  const int qx = d.qn[0], qy = d.qn[1];
  const int x = q % qx, y = (q / qx) % qy, z = q / (qx * qy);
  const int gx = (d.q0[0] + x) % d.gn[0], gy = (d.q0[1] + y) % d.gn[1], gz = (d.q0[2] + z) % d.gn[2];
  double v = v_extra ? v_extra[d.gvoff + ((long long)gz * d.gn[1] + gy) * d.gn[0] + gx] : 0.0;
  if (!isfinite(v)) atomicOr(&flags[k], EF_BAD);
  const double inv_rc2 = 1.0 / (r_cut * r_cut);
  for (int ai = 0; ai < d.pa_count; ai++) {
    const AtomBox& a = boxes[d.pa_begin + ai];
    int ix = x - a.s[0]; if (ix < 0) ix += qx;
    if (ix >= a.l[0]) continue;
    int iy = y - a.s[1]; if (iy < 0) iy += qy;
    if (iy >= a.l[1]) continue;
    int iz = z - a.s[2]; if (iz < 0) iz += d.qn[2];
    if (iz >= a.l[2]) continue;
    const double* t = dtab + a.toff;
    const double dx = t[ix], dy = t[a.l[0] + iy], dz = t[a.l[0] + a.l[1] + iz];
    const double d2 = dx * dx + dy * dy + dz * dz;
    const double u = 1.0 - d2 * inv_rc2;
    if (u > 0.0) v -= a.depth * exp(-d2 / (2.0 * a.wwidth * a.wwidth)) * u * u * u;
  }
  V64[d.voff + q] = v;
  V32[d.voff + q] = float(v);
}

void launch_setup_v(const BatchArgs& b, const AtomBox* boxes, const double* dtab, const double* v_extra, double r_cut,
                    double* V64, float* V32, int* flags, cudaStream_t st) {

  dim3 grid((g_max_points + 255) / 256, b.M);
  count_launch(); k_setup_v<<<grid, 256, 0, st>>>(b, boxes, dtab, v_extra, r_cut, V64, V32, flags);
}

// ---- SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator ----
// value(c) = (c+1)-th output for state `seed`; c = elem*2^40 + vec*2^24 + point.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long c) {
  unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void k_random_init(BatchArgs b, T* X, const long long* xo, unsigned long long seed) {
  const int k = blockIdx.z, v = blockIdx.y;
  const ElemDesc& d = b.desc[k];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n_blk || p >= d.N) return;
  const unsigned long long c = ((unsigned long long)k << 40) + ((unsigned long long)v << 24) + (unsigned long long)p;
  const unsigned long long z = splitmix64_at(seed, c);
  const double u = double(z >> 11) * 0x1.0p-53;
  X[xo[k] + (long long)v * d.N + p] = T(2.0 * u - 1.0);
}

template <typename T>
void launch_random_init(const BatchArgs& b, T* X, const long long* xo, unsigned long long seed, cudaStream_t st) {


  dim3 grid((g_max_points + 255) / 256, g_max_nblk, b.M);
  count_launch(); k_random_init<T><<<grid, 256, 0, st>>>(b, X, xo, seed);
}
thread_local int g_max_nblk = 0;

// ---- Chebyshev filter coefficients (scaled three-term recurrence) ----
// bounds[k] = {a0, b_low, b_up}; step 1: Y = (s1/e)(H - c)X;
// step i>1: s' = 1/(2/s1 - s), Y' = (2 s'/e)(H - c)Y - s s' Y_prev.
// Steps i >= pdeg[k] (when given) get alpha = 0, beta = 1: y_{i+1} = y_{i-1}, so that the element's block
// stays at y_{pdeg[k]} after the pass (D - pdeg[k] even) while the others run on.
__global__ void k_cheb_coeffs(BatchArgs b, const double* bounds, double* cheb, int degree, const int* pdeg) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.M) return;
  const double a0 = bounds[3 * k], bl = bounds[3 * k + 1], bu = bounds[3 * k + 2];
  const double e = 0.5 * (bu - bl), c = 0.5 * (bu + bl);
  double sigma = e / (a0 - c);
  const double sigma1 = sigma;
  double* ck = cheb + (long long)k * 3 * degree;
  ck[0] = sigma1 / e; ck[1] = c; ck[2] = 0.0;
  for (int i = 1; i < degree; i++) {
    const double sn = 1.0 / (2.0 / sigma1 - sigma);
    ck[3 * i] = 2.0 * sn / e;
    ck[3 * i + 1] = c;
    ck[3 * i + 2] = -sigma * sn;
    sigma = sn;
  }
  if (pdeg != nullptr)
    for (int i = max(1, pdeg[k]); i < degree; i++) {
      ck[3 * i] = 0.0;
      ck[3 * i + 1] = 0.0;
      ck[3 * i + 2] = 1.0;
    }
}
void launch_cheb_coeffs(const BatchArgs& b, const double* bounds, double* cheb, int degree, cudaStream_t st,
                        const int* pdeg) {
  count_launch(); k_cheb_coeffs<<<(b.M + 127) / 128, 128, 0, st>>>(b, bounds, cheb, degree, pdeg);
}

// Y = alpha (HX - c X) with the step-1 coefficients
template <typename T>
__global__ void k_cheb_first(BatchArgs b, const T* X, const T* HX, T* Y, const long long* xo, const double* cheb,
                             int cheb_stride) {
  const int k = blockIdx.z, v = blockIdx.y;
  if (!(b.flags == nullptr || (b.flags[k] & EF_ACTIVE))) return;
  const ElemDesc& d = b.desc[k];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n_blk || p >= d.N) return;
  const long long i = xo[k] + (long long)v * d.N + p;
  const T alpha = T(cheb[(long long)k * cheb_stride]), c = T(cheb[(long long)k * cheb_stride + 1]);
  Y[i] = alpha * (HX[i] - c * X[i]);
}
template <typename T>
void launch_cheb_first(const BatchArgs& b, const T* X, const T* HX, T* Y, const long long* xo, const double* cheb,
                       int cheb_stride, cudaStream_t st) {

  dim3 grid((g_max_points + 255) / 256, g_max_nblk, b.M);
  count_launch(); k_cheb_first<T><<<grid, 256, 0, st>>>(b, X, HX, Y, xo, cheb, cheb_stride);
}

// ---- block copy with type conversion between two packed layouts ----
template <typename TS, typename TD>
__global__ void k_convert(BatchArgs b, const TS* X, const long long* xo, TD* Y, const long long* yo, int nvec_mode) {
  const int k = blockIdx.z, v = blockIdx.y;
  const ElemDesc& d = b.desc[k];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvec_of(d, nvec_mode) || p >= d.N) return;
  Y[yo[k] + (long long)v * d.N + p] = TD(X[xo[k] + (long long)v * d.N + p]);
}
template <typename TS, typename TD>
void launch_convert(const BatchArgs& b, const TS* X, const long long* xo, TD* Y, const long long* yo, int nvec_mode,
                    cudaStream_t st) {

  dim3 grid((g_max_points + 255) / 256, nvec_mode == NV_ONE ? 1 : g_max_nblk, b.M);
  count_launch(); k_convert<TS, TD><<<grid, 256, 0, st>>>(b, X, xo, Y, yo, nvec_mode);
}

// ---- restriction of Q blocks to E ----
__global__ void k_restrict(BatchArgs b, const double* X, const long long* xo, double* XE, const long long* eo,
                           int nvec_mode) {
  const int k = blockIdx.z, v = blockIdx.y;
  const ElemDesc& d = b.desc[k];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvec_of(d, nvec_mode) || e >= d.NE) return;
  const int ex = e % d.en[0], ey = (e / d.en[0]) % d.en[1], ez = e / (d.en[0] * d.en[1]);
  const int q = ((ez + d.eo[2]) * d.qn[1] + (ey + d.eo[1])) * d.qn[0] + ex + d.eo[0];
  XE[eo[k] + (long long)v * d.NE + e] = X[xo[k] + (long long)v * d.N + q];
}
void launch_restrict(const BatchArgs& b, const double* X, const long long* xo, double* XE, const long long* eo,
                     int nvec_mode, cudaStream_t st) {

  dim3 grid((g_max_points + 255) / 256, g_max_nblk, b.M);
  count_launch(); k_restrict<<<grid, 256, 0, st>>>(b, X, xo, XE, eo, nvec_mode);
}

// ---- display sign: largest |entry| of each ALB positive (ties to the lowest index) ----
__global__ void k_alb_sign(BatchArgs b, double* A, const long long* ao, double* C, int ldc) {
  const int k = blockIdx.y, j = blockIdx.x;
  const ElemDesc& d = b.desc[k];
  if (j >= d.n_alb) return;
  double* Aj = A + ao[k] + (long long)j * d.NE;
  double best = -1.0;
  int bi = 0;
  bool first = true;
  for (int e = threadIdx.x; e < d.NE; e += blockDim.x) {
    const double a = fabs(Aj[e]);   // NaN entries never win (comparisons are false)
    if (first || a > best || (a == best && e < bi)) { best = isnan(a) ? -1.0 : a; bi = e; first = false; }
  }
  __shared__ double sb[256];
  __shared__ int si[256];
  sb[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = sb[threadIdx.x + s];
      const int oi = si[threadIdx.x + s];
      if (o > sb[threadIdx.x] || (o == sb[threadIdx.x] && oi < si[threadIdx.x])) {
        sb[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const int ibest = (si[0] >= 0 && si[0] < d.NE) ? si[0] : 0;
  const bool flip = Aj[ibest] < 0.0;
  __syncthreads();
  if (!flip) return;
  for (int e = threadIdx.x; e < d.NE; e += blockDim.x) Aj[e] = -Aj[e];
  double* Ck = C + (long long)k * ldc * ldc;
  for (int i = threadIdx.x; i < d.n_eig; i += blockDim.x) Ck[i * ldc + j] = -Ck[i * ldc + j];
}
void launch_alb_sign(const BatchArgs& b, double* A, const long long* ao, double* C, int ldc, cudaStream_t st) {

  dim3 grid(g_max_nalb, b.M);
  count_launch(); k_alb_sign<<<grid, 256, 0, st>>>(b, A, ao, C, ldc);
}
thread_local int g_max_nalb = 0;

// ---- convergence: residual norms, bounds for the next filter, active flags ----
// resid2[k][j] holds sum_p (HX_j - theta_j X_j)^2 dV-less; resid = sqrt(resid2 dV).  The stopping
// test is stage_converged (convergence.h): tol, and in the FP32 stage tol_mixed or stagnation at the
// FP32 rounding floor.
__global__ void k_update_convergence(BatchArgs b, const double* resid2, int ldr, double* resid, const double* theta,
                                     double* bounds, double tol, double tol_mixed, int mixed, double* prev_res,
                                     int* stall, int* flags, int* active_count, int* iters) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.M) return;
  if (!(flags[k] & EF_ACTIVE)) return;
  unsigned long long* hist_max = reinterpret_cast<unsigned long long*>(active_count + 2);
  const ElemDesc& d = b.desc[k];
  double mx = 0.0;
  for (int j = 0; j < d.n_blk; j++) {
    const double r = sqrt(fmax(resid2[k * ldr + j], 0.0) * d.dV);
    resid[k * ldr + j] = r;
    if (j < d.n_eig) mx = fmax(mx, r);
  }
  bounds[3 * k] = theta[k * ldr];
  bounds[3 * k + 1] = theta[k * ldr + d.n_blk - 1];
  iters[k] += 1;
  if (!isfinite(mx)) atomicOr(&flags[k], EF_BAD);
  const bool done = stage_converged(mx, tol, tol_mixed, mixed, bounds[3 * k + 2], &prev_res[k], &stall[k]) != 0;
  if (isfinite(mx)) atomicMax(hist_max, (unsigned long long)__double_as_longlong(mx));
  if (done) atomicAnd(&flags[k], ~EF_ACTIVE);
  else atomicAdd(active_count, 1);
}
// Filter degree of the next pass: the largest m <= max_degree for which the scaled Chebyshev polynomial's
// growth over the block's spectrum, |T_m(x(a0))| = cosh(m acosh|x(a0)|), stays within range_log
// (= acosh of the largest growth the precision carries), minimised over the active elements; one CTA.
__global__ void k_pass_degree(BatchArgs b, const double* bounds, int max_degree, double range_log, int* pdeg,
                              int* out) {
  __shared__ int red[256];
  auto cap = [&](int k) {
    const double a0 = bounds[3 * k], bl = bounds[3 * k + 1], bu = bounds[3 * k + 2];
    const double e = 0.5 * (bu - bl), c = 0.5 * (bu + bl);
    const double x = e > 0.0 ? fabs((a0 - c) / e) : 1.0;
    int m = max_degree;
    if (x > 1.0) {
      const double mk = floor(range_log / acosh(x));
      if (mk < double(m)) m = int(fmax(mk, 8.0));
    }
    return min(m, max_degree);
  };
  int m = 2;
  for (int k = threadIdx.x; k < b.M; k += blockDim.x)
    if (!b.flags || (b.flags[k] & EF_ACTIVE)) m = max(m, cap(k));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const int D = red[0];
  // an element stops after d_k steps with D - d_k even (the frozen recurrence alternates two vectors)
  for (int k = threadIdx.x; k < b.M; k += blockDim.x) {
    int dk = (!b.flags || (b.flags[k] & EF_ACTIVE)) ? cap(k) : D;
    dk -= (D - dk) & 1;
    pdeg[k] = max(dk, 2);
  }
  if (threadIdx.x == 0) *out = D;
}
void launch_pass_degree(const BatchArgs& b, const double* bounds, int max_degree, double range_log, int* pdeg,
                        int* out, cudaStream_t st) {
  count_launch(); k_pass_degree<<<1, 256, 0, st>>>(b, bounds, max_degree, range_log, pdeg, out);
}

void launch_update_convergence(const BatchArgs& b, const double* resid2, int ldr, double* resid, const double* theta,
                               double* bounds, double tol, double tol_mixed, int mixed, double* prev_res, int* stall,
                               int* flags, int* active_count, int* iters, cudaStream_t st) {
  count_launch(); k_update_convergence<<<(b.M + 127) / 128, 128, 0, st>>>(b, resid2, ldr, resid, theta, bounds, tol, tol_mixed, mixed,
                                                          prev_res, stall, flags, active_count, iters);
}

// ---- Lanczos upper bound: one vector per element at offsets o[k] ----
template <typename T>
__global__ void k_dot(BatchArgs b, const T* X, const T* Y, const long long* o, double* out, int ostride) {
  const int k = blockIdx.y;
  const ElemDesc& d = b.desc[k];
  double s = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < d.N; p += gridDim.x * blockDim.x)
    s += double(X[o[k] + p]) * double(Y[o[k] + p]);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(&out[(long long)k * ostride], s);
}
template <typename T>
void launch_dot(const BatchArgs& b, const T* X, const T* Y, const long long* o, double* out, int ostride,
                cudaStream_t st) {
  count_launch(); k_dot<T><<<dim3(32, b.M), 256, 0, st>>>(b, X, Y, o, out, ostride);
}

__global__ void k_store_sqrt(BatchArgs b, const double* src, double* dst, int stride) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < b.M) dst[(long long)k * stride] = sqrt(fmax(src[k], 0.0));
}
void launch_store_sqrt(const BatchArgs& b, const double* src, double* dst, int stride, cudaStream_t st) {
  count_launch(); k_store_sqrt<<<(b.M + 127) / 128, 128, 0, st>>>(b, src, dst, stride);
}

__global__ void k_final_resid(BatchArgs b, const double* resid2, int ldr, double* resid) {
  const int k = blockIdx.x;
  const ElemDesc& d = b.desc[k];
  for (int j = threadIdx.x; j < d.n_blk; j += blockDim.x)
    resid[k * ldr + j] = sqrt(fmax(resid2[k * ldr + j], 0.0) * d.dV);
}
void launch_final_resid(const BatchArgs& b, const double* resid2, int ldr, double* resid, cudaStream_t st) {
  count_launch(); k_final_resid<<<b.M, 128, 0, st>>>(b, resid2, ldr, resid);
}

__global__ void k_set_active(BatchArgs b, int* flags) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < b.M) flags[k] |= EF_ACTIVE;
}
void launch_set_active(const BatchArgs& b, int* flags, cudaStream_t st) {
  count_launch(); k_set_active<<<(b.M + 127) / 128, 128, 0, st>>>(b, flags);
}

// per-element status: bad input > Cholesky failure > not converged (hit_cap) > ok
__global__ void k_elem_status(BatchArgs b, const int* flags, const double* resid, int ldr, double tol,
                              const int* hit_cap, int* status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.M) return;
  int s = ST_OK;
  if (hit_cap && hit_cap[k]) s = ST_NOT_CONVERGED;
  if (flags[k] & EF_CHOL_FAIL) s = ST_CHOLESKY_FAIL;
  if (flags[k] & EF_BAD) s = ST_BAD_INPUT;
  for (int j = 0; j < b.desc[k].n_eig; j++)
    if (!isfinite(resid[k * ldr + j])) s = ST_BAD_INPUT;
  status[k] = s;
}
void launch_elem_status(const BatchArgs& b, const int* flags, const double* resid, int ldr, double tol,
                        const int* hit_cap, int* status, cudaStream_t st) {
  count_launch(); k_elem_status<<<(b.M + 127) / 128, 128, 0, st>>>(b, flags, resid, ldr, tol, hit_cap, status);
}

// f <- f - alpha v - beta_prev v_old
template <typename T>
__global__ void k_lanczos_update(BatchArgs b, T* v, T* f, T* vold, const long long* o, const double* alpha,
                                 const double* beta_prev, int stride, int first) {
  const int k = blockIdx.y;
  const ElemDesc& d = b.desc[k];
  const double a = alpha[(long long)k * stride], bp = first ? 0.0 : beta_prev[(long long)k * stride];
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < d.N; p += gridDim.x * blockDim.x) {
    double fv = double(f[o[k] + p]) - a * double(v[o[k] + p]);
    if (!first) fv -= bp * double(vold[o[k] + p]);
    f[o[k] + p] = T(fv);
  }
}
template <typename T>
void launch_lanczos_update(const BatchArgs& b, T* v, T* f, T* vold, const long long* o, const double* alpha,
                           const double* beta_prev, int stride, int first, cudaStream_t st) {
  count_launch(); k_lanczos_update<T><<<dim3(32, b.M), 256, 0, st>>>(b, v, f, vold, o, alpha, beta_prev, stride, first);
}

// v_old <- v (if vold != null);  v <- f / sqrt(nrm2)
template <typename T>
__global__ void k_scale_vec(BatchArgs b, T* v, const T* f, T* vold, const long long* o, const double* nrm2) {
  const int k = blockIdx.y;
  const ElemDesc& d = b.desc[k];
  const double s = nrm2[k] > 0.0 ? 1.0 / sqrt(nrm2[k]) : 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < d.N; p += gridDim.x * blockDim.x) {
    if (vold) vold[o[k] + p] = v[o[k] + p];
    v[o[k] + p] = T(double(f[o[k] + p]) * s);
  }
}
template <typename T>
void launch_scale_vec_old(const BatchArgs& b, T* v, const T* f, T* vold, const long long* o, const double* nrm2,
                          cudaStream_t st) {
  count_launch(); k_scale_vec<T><<<dim3(32, b.M), 256, 0, st>>>(b, v, f, vold, o, nrm2);
}

// largest eigenvalue of the Lanczos tridiagonal (bisection on Sturm counts) + |f|
__global__ void k_lanczos_bound(BatchArgs b, const double* alphas, const double* betas, int steps,
                                const double* fnorm2, double* bounds, double* lanczos_min) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.M) return;
  const double* al = alphas + (long long)k * steps;
  const double* be = betas + (long long)k * steps;  // be[j] couples j-1 and j (j >= 1)
  double lo = 1e300, hi = -1e300;
  for (int j = 0; j < steps; j++) {
    const double r = (j > 0 ? fabs(be[j]) : 0.0) + (j + 1 < steps ? fabs(be[j + 1]) : 0.0);
    lo = fmin(lo, al[j] - r);
    hi = fmax(hi, al[j] + r);
  }
  // count of eigenvalues < x via the LDL^T pivots (Sturm sequence)
  auto count_below = [&](double x) {
    int cnt = 0;
    double q = 1.0;
    for (int j = 0; j < steps; j++) {
      const double bb = j > 0 ? be[j] * be[j] : 0.0;
      q = (al[j] - x) - (j > 0 ? bb / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0.0) cnt++;
    }
    return cnt;
  };
  const double lo0 = lo, hi0 = hi;
  for (int it = 0; it < 200; it++) {   // largest Ritz value
    const double x = 0.5 * (lo + hi);
    if (count_below(x) >= steps) hi = x; else lo = x;
  }
  bounds[3 * k + 2] = hi + sqrt(fmax(fnorm2[k], 0.0));
  lo = lo0; hi = hi0;
  for (int it = 0; it < 200; it++) {   // smallest Ritz value
    const double x = 0.5 * (lo + hi);
    if (count_below(x) >= 1) hi = x; else lo = x;
  }
  lanczos_min[k] = lo;
}
void launch_lanczos_bound(const BatchArgs& b, const double* alphas, const double* betas, int steps,
                          const double* fnorm2, double* bounds, double* lanczos_min, cudaStream_t st) {
  count_launch(); k_lanczos_bound<<<(b.M + 127) / 128, 128, 0, st>>>(b, alphas, betas, steps, fnorm2, bounds,
                                                                     lanczos_min);
}

// first filter pass: scale at min(start-up Ritz minimum, Lanczos minimum) so that components below the
// start block's Ritz values cannot be amplified beyond the FP32 range
__global__ void k_first_a0(BatchArgs b, const double* lanczos_min, double* bounds) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < b.M) bounds[3 * k] = fmin(bounds[3 * k], lanczos_min[k]);
}
void launch_first_a0(const BatchArgs& b, const double* lanczos_min, double* bounds, cudaStream_t st) {
  count_launch(); k_first_a0<<<(b.M + 127) / 128, 128, 0, st>>>(b, lanczos_min, bounds);
}

template void launch_random_init<float>(const BatchArgs&, float*, const long long*, unsigned long long, cudaStream_t);
template void launch_random_init<double>(const BatchArgs&, double*, const long long*, unsigned long long, cudaStream_t);
template void launch_cheb_first<float>(const BatchArgs&, const float*, const float*, float*, const long long*,
                                       const double*, int, cudaStream_t);
template void launch_cheb_first<double>(const BatchArgs&, const double*, const double*, double*, const long long*,
                                        const double*, int, cudaStream_t);
template void launch_convert<float, double>(const BatchArgs&, const float*, const long long*, double*,
                                            const long long*, int, cudaStream_t);
template void launch_convert<double, double>(const BatchArgs&, const double*, const long long*, double*,
                                             const long long*, int, cudaStream_t);
template void launch_convert<float, float>(const BatchArgs&, const float*, const long long*, float*, const long long*,
                                           int, cudaStream_t);
template void launch_convert<double, float>(const BatchArgs&, const double*, const long long*, float*,
                                            const long long*, int, cudaStream_t);
template void launch_dot<float>(const BatchArgs&, const float*, const float*, const long long*, double*, int,
                                cudaStream_t);
template void launch_dot<double>(const BatchArgs&, const double*, const double*, const long long*, double*, int,
                                 cudaStream_t);
template void launch_lanczos_update<float>(const BatchArgs&, float*, float*, float*, const long long*, const double*,
                                           const double*, int, int, cudaStream_t);
template void launch_lanczos_update<double>(const BatchArgs&, double*, double*, double*, const long long*,
                                            const double*, const double*, int, int, cudaStream_t);
template void launch_scale_vec_old<float>(const BatchArgs&, float*, const float*, float*, const long long*,
                                          const double*, cudaStream_t);
template void launch_scale_vec_old<double>(const BatchArgs&, double*, const double*, double*, const long long*,
                                           const double*, cudaStream_t);

}  // namespace dgdft
