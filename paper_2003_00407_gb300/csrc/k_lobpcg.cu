// Element-wise kernels of the LOBPCG local solver (Alg. LOBPCG, Eqs. 3-5) with the Teter preconditioner;
// the H applications, transforms, Gram matrices and the projected generalized eigenproblem reuse the
// kernels of the CheFSI path.  FP64, all elements at once (per-element blocks of n vectors).
#include "kernels.h"

namespace dgdft {

__device__ __forceinline__ int lob_nvec(const ElemDesc& d) { return d.n_blk; }

// R = HX - theta X into W (row v of element k), squared residual norms (without dV) into resid2[k*ld + v]
__global__ void k_lobpcg_resid(BatchArgs b, const double* X, const double* HX, const long long* xo,
                               const double* theta, int ld, double* W, double* resid2) {
  const int k = blockIdx.z, v = blockIdx.y;
  if (!(b.flags == nullptr || (b.flags[k] & EF_ACTIVE))) return;
  const ElemDesc& d = b.desc[k];
  if (v >= lob_nvec(d)) return;
  const double th = theta[(long long)k * ld + v];
  const long long o = xo[k] + (long long)v * d.N;
  double s = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < d.N; p += gridDim.x * blockDim.x) {
    const double r = HX[o + p] - th * X[o + p];
    W[o + p] = r;
    s += r * r;
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(&resid2[(long long)k * ld + v], s);
}

// out[k*ld + v] = dV sum_p X[v][p] Y[v][p] (callers zero out first)
__global__ void k_vec_dots(BatchArgs b, const double* X, const double* Y, const long long* xo, int ld, double* out) {
  const int k = blockIdx.z, v = blockIdx.y;
  if (!(b.flags == nullptr || (b.flags[k] & EF_ACTIVE))) return;
  const ElemDesc& d = b.desc[k];
  if (v >= lob_nvec(d)) return;
  const long long o = xo[k] + (long long)v * d.N;
  double s = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < d.N; p += gridDim.x * blockDim.x) s += X[o + p] * Y[o + p];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(&out[(long long)k * ld + v], s * d.dV);
}

// X' = X C_X + W C_W + P C_P, P' = W C_W + P C_P (Eq. 4 and the conjugate direction), and the same for
// the H-images; C [ld][ld] per element, row blocks X (0..n), W (n..2n), P (2n..3n; absent when nb == 2)
__global__ void k_lobpcg_update(BatchArgs b, const long long* xo, const double* C, int ld, int nb, const double* X,
                                const double* W, const double* P, const double* HX, const double* HW,
                                const double* HP, double* Xn, double* Pn, double* HXn, double* HPn) {
  const int k = blockIdx.z, j = blockIdx.y;
  const ElemDesc& d = b.desc[k];
  const int n = lob_nvec(d);
  if (j >= n) return;
  if (!(b.flags == nullptr || (b.flags[k] & EF_ACTIVE))) {
    // a converged element keeps its blocks (the caller swaps the new and old buffers)
    const long long o = xo[k] + (long long)j * d.N;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < d.N; p += gridDim.x * blockDim.x) {
      Xn[o + p] = X[o + p];
      HXn[o + p] = HX[o + p];
      if (nb == 3) {
        Pn[o + p] = P[o + p];
        HPn[o + p] = HP[o + p];
      }
    }
    return;
  }
  __shared__ double cj[3 * 96];
  const double* Ck = C + (long long)k * ld * ld;
  for (int i = threadIdx.x; i < nb * n; i += blockDim.x) cj[i] = Ck[(long long)i * ld + j];
  __syncthreads();
  const long long ok = xo[k];
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < d.N; p += gridDim.x * blockDim.x) {
    double x = 0.0, hx = 0.0, pw = 0.0, hpw = 0.0;
    for (int i = 0; i < n; i++) {
      const long long o = ok + (long long)i * d.N + p;
      x = fma(cj[i], X[o], x);
      hx = fma(cj[i], HX[o], hx);
      pw = fma(cj[n + i], W[o], pw);
      hpw = fma(cj[n + i], HW[o], hpw);
      if (nb == 3) {
        pw = fma(cj[2 * n + i], P[o], pw);
        hpw = fma(cj[2 * n + i], HP[o], hpw);
      }
    }
    const long long oj = ok + (long long)j * d.N + p;
    Xn[oj] = x + pw;
    HXn[oj] = hx + hpw;
    Pn[oj] = pw;
    HPn[oj] = hpw;
  }
}

// rows of X (and of Y when given) divided by sqrt(nrm2[k*ld + v]) (unit dV-norm rows of the trial blocks)
__global__ void k_scale_rows(BatchArgs b, double* X, double* Y, const long long* xo, const double* nrm2, int ld) {
  const int k = blockIdx.z, v = blockIdx.y;
  if (!(b.flags == nullptr || (b.flags[k] & EF_ACTIVE))) return;
  const ElemDesc& d = b.desc[k];
  if (v >= lob_nvec(d)) return;
  const double q = nrm2[(long long)k * ld + v];
  const double s = q > 0.0 ? 1.0 / sqrt(q) : 0.0;
  const long long o = xo[k] + (long long)v * d.N;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < d.N; p += gridDim.x * blockDim.x) {
    X[o + p] *= s;
    if (Y) Y[o + p] *= s;
  }
}

void launch_scale_rows(const BatchArgs& b, double* X, double* Y, const long long* xo, const double* nrm2, int ld,
                       cudaStream_t st) {
  count_launch();
  k_scale_rows<<<dim3(16, g_max_nblk, b.M), 256, 0, st>>>(b, X, Y, xo, nrm2, ld);
}

void launch_lobpcg_resid(const BatchArgs& b, const double* X, const double* HX, const long long* xo,
                         const double* theta, int ld, double* W, double* resid2, cudaStream_t st) {
  count_launch();
  k_lobpcg_resid<<<dim3(16, g_max_nblk, b.M), 256, 0, st>>>(b, X, HX, xo, theta, ld, W, resid2);
}

void launch_vec_dots(const BatchArgs& b, const double* X, const double* Y, const long long* xo, int ld, double* out,
                     cudaStream_t st) {
  count_launch();
  k_vec_dots<<<dim3(16, g_max_nblk, b.M), 256, 0, st>>>(b, X, Y, xo, ld, out);
}

void launch_lobpcg_update(const BatchArgs& b, const long long* xo, const double* C, int ld, int nb, const double* X,
                          const double* W, const double* P, const double* HX, const double* HW, const double* HP,
                          double* Xn, double* Pn, double* HXn, double* HPn, cudaStream_t st) {
  count_launch();
  k_lobpcg_update<<<dim3((g_max_points + 255) / 256, g_max_nblk, b.M), 256, 0, st>>>(b, xo, C, ld, nb, X, W, P, HX,
                                                                                     HW, HP, Xn, Pn, HXn, HPn);
}

}  // namespace dgdft
